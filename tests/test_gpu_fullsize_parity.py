"""Bit-exact GPU parity of the circuits at the 128-element sizes, and parity of the
library's own constants with the oracle's.

With the oracle's keys, input ciphertexts, mask encodings and indicator coefficients
imported, every CUDA circuit below returns the oracle's ciphertext bit for bit:

* the 128-element rank (Alg. 3) on the n = 2^16, 28 + 3 limb set the benchmark times;
* on an n = 2^15 ring (the smallest that holds a 128 x 128 matrix), 34 + 3 limbs,
  comparator g^3 f^2, values on a 64-level grid (ties): argmin with the tie-corrected
  ranks (Alg. 4 + Alg. 6) on a three-member stack (the depth-first Paterson-Stockmeyer
  recursion of wide stacks, 1024 indicator coefficients), argmax with every tied
  maximum (Cmp_GE of Sec. 3.2), the sort (Alg. 5, column form), the blocked rank of
  two blocks of 128 (Alg. 7, Eq. 3), and two slot-packed 64-element ranks (Q = 2);
* the n = 2^16 set's mask encodings, and the indicator and Chebyshev-comparator
  coefficients, as the library computes them (no import), against the oracle's:
  within one unit per scaled coefficient and 1e-12 per coefficient;
* an 8-element rank, argmin and sort with the library's own encodings and
  coefficients (nothing imported) decrypt to the oracle's values.

The oracle work here takes minutes of host time (marked slow).
"""
import numpy as np
import pytest

from oracle import ckks, circuits as C
from paper_2412_15126_gb300 import inputs
from tests import helpers

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def rank_rotations(N):
    """The rotation amounts of a rank (ReplR, TransR, ReplC, SumR), with the sums of
    the step pairs its chains take two at a time."""
    k = int(np.log2(N))
    chains = [[-(N << i) for i in range(k)], [-(1 << i) for i in range(k)], [N << i for i in range(k)],
              [-((N * (N - 1)) >> i) for i in range(1, k + 1)]]
    rs = set()
    for ch in chains:   # every step, and the sums of the step pairs taken two at a time
        rs.update(ch)
        rs.update(ch[i] + ch[i + 1] for i in range(0, len(ch) - 1, 2))
    return sorted(rs)


# --------------------------------------------------------------------------
# The 128-element rank on the benchmark's parameter set
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg2():
    P = helpers.oracle_params("cfg2")
    keys = ckks.keygen(P, 2412, helpers.galois_elts(P, rank_rotations(128)))
    ctx = helpers.gpu_context("cfg2")
    helpers.import_keys(ctx, keys)
    yield P, keys, ctx
    ctx.close()


def test_cfg2_library_encodings_match_the_oracle(cfg2):
    """The library's own mask encodings (its FFT) against the oracle's encoder: the
    plaintexts differ by at most one unit per coefficient at the top level's scale."""
    from paper_2412_15126_gb300 import rankfhe
    P, _, ctx = cfg2
    s = ckks.scalar_scale(P, P.L)
    for kind in helpers.ALL_MASKS:
        mine = ctx.encoding_export(helpers.MASK_IDS[kind], 128, 1, 0)
        ref = ckks.encode_unscaled(C.mask_slots(kind, 128, 1, slots=P.slots), P.n)
        assert np.max(np.abs(ckks.rha(s * mine) - ckks.rha(s * ref))) <= 1, kind
    mine = ctx.encoding_export(rankfhe.MASK_VALID, 128, 1, 100)
    ref = ckks.encode_unscaled(C.mask_slots("valid", 128, 1, 100, slots=P.slots), P.n)
    assert np.max(np.abs(ckks.rha(s * mine) - ckks.rha(s * ref))) <= 1


def test_cfg2_library_indicator_coefficients_match_the_oracle(cfg2):
    _, _, ctx = cfg2
    for N in (8, 128, 512):
        mine = ctx.indicator_export(N)
        ref = C.sinc2_window_coeffs(N)
        assert mine.shape == ref.shape
        assert np.max(np.abs(mine - ref)) < 1e-12, N


def test_cfg2_rank_n128_bit_exact(cfg2):
    P, keys, ctx = cfg2
    helpers.import_encodings(ctx, P, 128, kinds=("row0", "col0"))
    v = inputs.gap_vector(128, 2.0 ** -9, 5)
    ct = ckks.encrypt(P, keys, v, 5)
    R = C.rank(C.OracleCkks(P, keys), ct, 128, 4, 2)
    g = ctx.rank(ctx.ct_import(ct.c, ct.level, N=128))
    assert g.level == R.level == P.L - 20
    assert np.array_equal(g.export(), R.c)
    assert np.max(np.abs(ctx.decrypt(g) - C.brute_fractional_rank(v))) < 0.25


# --------------------------------------------------------------------------
# Order statistics, sort, blocked rank and slot packing at N = 128 (n = 2^15)
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def big():
    P = helpers.oracle_params("big15")
    rots = sorted(set(helpers.rotation_set(128)) | set(rank_rotations(64)))
    keys = ckks.keygen(P, 2413, helpers.galois_elts(P, rots))
    ctx = helpers.gpu_context("big15")
    helpers.import_keys(ctx, keys)
    helpers.import_encodings(ctx, P, 128, kinds=helpers.ALL_MASKS)
    helpers.import_encodings(ctx, P, 64, Q=2, kinds=("row0", "col0"))
    ctx.indicator_import(128, C.sinc2_window_coeffs(128))
    yield P, keys, ctx
    ctx.close()


def _grid(seed, N=128):
    return inputs.grid_vector(N, 64, seed)


def test_big_argmin_stack_of_three_bit_exact(big):
    """argmin (tie-corrected ranks, one-hot at the first minimum) of a three-member stack
    [a, b, a]: each member equals the oracle's circuit on its input."""
    from paper_2412_15126_gb300 import rankfhe
    P, keys, ctx = big
    va, vb = _grid(1), _grid(2)
    ca, cb = ckks.encrypt(P, keys, va, 11), ckks.encrypt(P, keys, vb, 12)
    B = C.OracleCkks(P, keys)
    ra = C.order_statistic(B, ca, 128, 1, 3, 2)
    rb = C.order_statistic(B, cb, 128, 1, 3, 2)
    ga, gb = ctx.ct_import(ca.c, ca.level, N=128), ctx.ct_import(cb.c, cb.level, N=128)
    parts = ctx.unstack(ctx.order_stat(ctx.stack([ga, gb, ga]), 1, rankfhe.TIES_FIRST))
    for part, ref in zip(parts, (ra, rb, ra)):
        assert part.level == ref.level
        assert np.array_equal(part.export(), ref.c)
    for part, v in zip(parts, (va, vb)):
        first = np.zeros(128)
        first[int(np.argmin(v))] = 1
        assert np.max(np.abs(ctx.decrypt(part) - first)) < 0.01


def test_big_argmax_all_ties_bit_exact(big):
    from paper_2412_15126_gb300 import rankfhe
    P, keys, ctx = big
    v = _grid(3)
    ct = ckks.encrypt(P, keys, v, 13)
    ref = C.order_statistic(C.OracleCkks(P, keys), ct, 128, 128, 3, 2, ties="all")
    g = ctx.order_stat(ctx.ct_import(ct.c, ct.level, N=128), 128, rankfhe.TIES_ALL)
    assert np.array_equal(g.export(), ref.c)
    assert np.max(np.abs(ctx.decrypt(g) - (v == v.max()))) < 0.01


def test_big_sort_bit_exact(big):
    P, keys, ctx = big
    v = _grid(4)
    ct = ckks.encrypt(P, keys, v, 14)
    ref = C.sort(C.OracleCkks(P, keys), ct, 128, 3, 2)
    g = ctx.sort(ctx.ct_import(ct.c, ct.level, N=128))
    assert g.level == ref.level
    assert np.array_equal(g.export(), ref.c)
    assert np.max(np.abs(ctx.decrypt(g) - np.sort(v))) < 0.01


def test_big_blocked_rank_two_blocks_of_128_bit_exact(big):
    P, keys, ctx = big
    v = inputs.gap_vector(256, 2.0 ** -9, 15)
    cts = [ckks.encrypt(P, keys, v[128 * i: 128 * (i + 1)], 15 + i) for i in range(2)]
    ref = C.rank_blocked(C.OracleCkks(P, keys), cts, 128, 3, 2)
    got = ctx.rank_blocked([ctx.ct_import(c.c, c.level, N=128) for c in cts])
    for g, r in zip(got, ref):
        assert g.level == r.level
        assert np.array_equal(g.export(), r.c)
    ranks = np.concatenate([ctx.decrypt(g) for g in got])
    assert np.max(np.abs(ranks - C.brute_fractional_rank(v))) < 0.25


def test_big_slot_packed_two_queries_bit_exact(big):
    """Two 64-element queries packed in one ciphertext (slots q 64^2 + j)."""
    P, keys, ctx = big
    v = np.concatenate([inputs.gap_vector(64, 2.0 ** -9, 16), inputs.gap_vector(64, 2.0 ** -9, 17)])
    z = np.zeros(P.slots)
    z[:64] = v[:64]
    z[64 * 64: 64 * 64 + 64] = v[64:]
    ct = ckks.encrypt(P, keys, z, 16)
    ref = C.rank(C.OracleCkks(P, keys), ct, 64, 3, 2, Q=2)
    g = ctx.rank(ctx.ct_import(ct.c, ct.level, N=64, Q=2))
    assert np.array_equal(g.export(), ref.c)
    got = ctx.decrypt(g)
    want = np.concatenate([C.brute_fractional_rank(v[:64]), C.brute_fractional_rank(v[64:])])
    assert np.max(np.abs(got - want)) < 0.25


# --------------------------------------------------------------------------
# Nothing imported: the library's own encoder and coefficients end to end
# --------------------------------------------------------------------------
def test_library_constants_end_to_end_n8():
    """rank, argmin and sort of 8 elements with the library's own mask encodings and
    indicator coefficients (only keys and input imported) decrypt to the same slot
    values as the oracle's circuits (which differ in the plaintexts' last units at most)."""
    from paper_2412_15126_gb300 import rankfhe
    P = helpers.oracle_params("ord")
    keys = ckks.keygen(P, 33, helpers.galois_elts(P, helpers.rotation_set(8)))
    ctx = helpers.gpu_context("ord")
    try:
        helpers.import_keys(ctx, keys)
        v = np.array([3, 1, 3, 0, 2, 1, 3, 2]) / 4.0
        ct = ckks.encrypt(P, keys, v, 21)
        B = C.OracleCkks(P, keys)
        g = ctx.ct_import(ct.c, ct.level, N=8)
        cases = [
            (ctx.rank(g), C.rank(B, ct, 8, 2, 1)),
            (ctx.order_stat(g, 1, rankfhe.TIES_FIRST), C.order_statistic(B, ct, 8, 1, 2, 1)),
            (ctx.sort(g), C.sort(B, ct, 8, 2, 1)),
        ]
        for got, ref in cases:
            assert got.level == ref.level
            assert np.max(np.abs(ctx.decrypt_slots(got) - ckks.decrypt(P, keys, ref))) < 1e-6
    finally:
        ctx.close()


def test_library_chebyshev_comparator_coefficients():
    for count in (16, 128, 2048):
        ctx = helpers.gpu_context("small", cmp_cheb=count)
        try:
            mine = ctx.comparator_export()
            ref = C.ChebCmp(count).coeffs
            assert mine.shape == ref.shape
            assert np.max(np.abs(mine - ref)) < 1e-12, count
        finally:
            ctx.close()
