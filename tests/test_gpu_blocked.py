"""GPU parity of the multi-ciphertext circuits with tie correction: blocked ranks
(Alg. 7 with Alg. 6 across blocks), the blocked order statistic (Alg. 4) and the
blocked sort (Alg. 8).

* n = 2^11, 24 limbs, blocks of 4 (a ring the oracle runs in seconds): with the
  oracle's keys, blocks, mask encodings and indicator imported, every output block
  equals the oracle's ciphertext bit for bit.
* n = 2^16, 34 limbs, N = 128 as two blocks of 64 on a 64-level grid (ties): the
  library's own keys, decrypted against the brute-force answers.
"""
import numpy as np
import pytest

from oracle import ckks, circuits as C
from paper_2412_15126_gb300 import inputs
from tests import helpers

pytestmark = pytest.mark.gpu

BSZ = 4


@pytest.fixture(scope="module")
def ordb():
    P = helpers.oracle_params("ordb")
    keys = ckks.keygen(P, 41, helpers.galois_elts(P, helpers.rotation_set(BSZ)))
    ctx = helpers.gpu_context("ordb")
    helpers.import_keys(ctx, keys)
    helpers.import_encodings(ctx, P, BSZ, kinds=("row0", "col0", "tie"))
    for L in (2, 3):
        D = L * BSZ
        for kind in ("row0s", "rowidx"):
            u = ckks.encode_unscaled(C.mask_slots(kind, BSZ, 1, D, slots=P.slots), P.n)
            ctx.encoding_import(helpers.MASK_IDS[kind], BSZ, 1, D, u)
        ctx.indicator_import(D, C.sinc2_window_coeffs(D))
    yield P, keys, ctx
    ctx.close()


def _encrypt_blocks(P, keys, ctx, v, seed):
    cts = [ckks.encrypt(P, keys, v[i * BSZ:(i + 1) * BSZ], seed + i) for i in range(len(v) // BSZ)]
    return cts, [ctx.ct_import(c.c, c.level, N=BSZ) for c in cts]


def test_blocked_tie_corrected_rank_bit_exact(ordb):
    from paper_2412_15126_gb300 import rankfhe
    P, keys, ctx = ordb
    v = np.array([3, 1, 3, 0, 2, 1, 3, 2, 0, 1, 2, 3]) / 8.0
    cts, g = _encrypt_blocks(P, keys, ctx, v, 10)
    ref, _ = C.rank_blocked_tc(C.OracleCkks(P, keys), cts, BSZ, 1, 1)
    got = ctx.rank_blocked(g, rankfhe.TIES_CORRECT)
    for a, b in zip(got, ref):
        assert a.level == b.level
        assert np.array_equal(a.export(), b.c)


def test_blocked_order_statistic_bit_exact(ordb):
    P, keys, ctx = ordb
    v = np.array([3, 1, 3, 0, 2, 0, 3, 2]) / 8.0
    cts, g = _encrypt_blocks(P, keys, ctx, v, 20)
    ref = C.order_statistic_blocked(C.OracleCkks(P, keys), cts, BSZ, 2, 1, 1)
    got = ctx.order_stat_blocked(g, 2)
    for a, b in zip(got, ref):
        assert np.array_equal(a.export(), b.c)


def test_blocked_sort_bit_exact(ordb):
    P, keys, ctx = ordb
    v = np.array([0.75, 0.125, 0.5, 0.0, 0.625, 0.25, 0.875, 0.375])
    cts, g = _encrypt_blocks(P, keys, ctx, v, 30)
    ref = C.sort_blocked(C.OracleCkks(P, keys), cts, BSZ, 1, 1)
    got = ctx.sort_blocked(g)
    for a, b in zip(got, ref):
        assert a.level == b.level
        assert np.array_equal(a.export(), b.c)


@pytest.fixture(scope="module")
def cfg3():
    ctx = helpers.gpu_context("cfg3")
    ctx.keygen(78, 64)
    yield ctx
    ctx.close()


def test_cfg3_blocked_two_by_64_with_ties(cfg3):
    from paper_2412_15126_gb300 import rankfhe
    ctx = cfg3
    v = inputs.grid_vector(128, 64, 9)
    blocks = [ctx.encrypt(v[:64], N=64), ctx.encrypt(v[64:], N=64)]
    R = np.concatenate([ctx.decrypt(r) for r in ctx.rank_blocked(blocks, rankfhe.TIES_CORRECT)])
    assert np.max(np.abs(R - C.brute_tie_corrected_rank(v))) < 0.05
    O = np.concatenate([ctx.decrypt(o) for o in ctx.order_stat_blocked(blocks, 1)])
    first = np.zeros(128)
    first[int(np.argmin(v))] = 1
    assert np.max(np.abs(O - first)) < 0.01
    S = np.concatenate([ctx.decrypt(s) for s in ctx.sort_blocked(blocks)])
    assert np.max(np.abs(S - np.sort(v))) < 0.01


def test_blocked_stacked_queries_identical_to_alone(ordb):
    """Blocks given as stacks (block i of two queries) return, per query, exactly the
    blocks of that query's circuit alone: rank (both forms), order statistic, sort."""
    from paper_2412_15126_gb300 import rankfhe
    P, keys, ctx = ordb
    vs = [np.array([3, 1, 3, 0, 2, 1, 3, 2]) / 8.0, np.array([0.75, 0.125, 0.5, 0.0, 0.625, 0.25, 0.875, 0.375])]
    qs = [_encrypt_blocks(P, keys, ctx, v, 40 + 10 * i)[1] for i, v in enumerate(vs)]
    stacked = [ctx.stack([q[b] for q in qs]) for b in range(2)]
    runs = [
        (lambda bl: ctx.rank_blocked(bl)),
        (lambda bl: ctx.rank_blocked(bl, rankfhe.TIES_CORRECT)),
        (lambda bl: ctx.order_stat_blocked(bl, 3)),
        (lambda bl: ctx.sort_blocked(bl)),
    ]
    for run in runs:
        together = run(stacked)
        for qi, q in enumerate(qs):
            alone = run(q)
            for b in range(2):
                assert np.array_equal(ctx.unstack(together[b])[qi].export(), alone[b].export())


def test_block_stacking_option_changes_nothing(ordb):
    """The plain per-query form (every block and pair ciphertext on its own) returns
    the stacked form's blocks bit for bit."""
    from paper_2412_15126_gb300 import rankfhe
    P, keys, ctx = ordb
    v = np.array([0.75, 0.125, 0.5, 0.0, 0.625, 0.25, 0.875, 0.375, 0.3125, 0.5625, 0.1875, 0.9375])
    _, g = _encrypt_blocks(P, keys, ctx, v, 60)
    stacked = [b.export() for b in ctx.rank_blocked(g)]
    ctx.set_option(rankfhe.OPT_BLOCK_STACKING, 0)
    try:
        plain = [b.export() for b in ctx.rank_blocked(g)]
    finally:
        ctx.set_option(rankfhe.OPT_BLOCK_STACKING, 1)
    for a, b in zip(stacked, plain):
        assert np.array_equal(a, b)


def test_blocked_rank_in_parts_bit_exact(ordb):
    """Alg. 7 with the block pairs divided in two parts (rk_rank_blocked_partial), the
    partial sums added (rk_add) and assembled (rk_rank_blocked_finish): bit for bit the
    oracle's blocked rank; the distributed helper with one rank gives the same."""
    from paper_2412_15126_gb300 import blocked_dist
    P, keys, ctx = ordb
    v = np.array([0.75, 0.125, 0.5, 0.0, 0.625, 0.25, 0.875, 0.375, 0.3125, 0.5625, 0.1875, 0.9375])
    cts, g = _encrypt_blocks(P, keys, ctx, v, 70)
    ref = C.rank_blocked(C.OracleCkks(P, keys), cts, BSZ, 1, 1)
    parts = blocked_dist.pair_partition(3, 2)
    A0, B0 = ctx.rank_blocked_partial(g, parts[0])
    A1, B1 = ctx.rank_blocked_partial(g, parts[1])
    got = ctx.rank_blocked_finish([ctx.add(a, b) for a, b in zip(A0, A1)], [ctx.add(a, b) for a, b in zip(B0, B1)])
    for a, b in zip(got, ref):
        assert a.level == b.level
        assert np.array_equal(a.export(), b.c)
    one = blocked_dist.blocked_rank_distributed(blocked_dist.CudaEvaluator(ctx, BSZ), g, 0, 1)
    for a, b in zip(one, ref):
        assert np.array_equal(a.export(), b.c)
    # the exchange form: a part's sums exported and imported again change nothing
    ev = blocked_dist.CudaEvaluator(ctx, BSZ)
    back = [ev.import_(ev.export(a), a) for a in A1]
    for a, b in zip(back, A1):
        assert np.array_equal(a.export(), b.export())


def _plain_blocks(P, v, f):
    """Row 0 of every block of f's output in the noiseless slot model."""
    Bp = C.PlainSlots(P.slots, P.L)
    out = f(Bp, [Bp.fresh(v[i * BSZ:(i + 1) * BSZ]) for i in range(len(v) // BSZ)])
    return np.concatenate([Bp.values(x)[:BSZ] for x in out])


@pytest.fixture(scope="module")
def ordb_packed():
    """The n = 2^11 ring with the keys of the tile-packing rotations too: 64 tiles of
    16 slots a ciphertext, rotations by +-16 2^s."""
    P = helpers.oracle_params("ordb")
    tile = BSZ * BSZ
    tiles = P.slots // tile
    rots = list(helpers.rotation_set(BSZ))
    s = 1
    while s < tiles:
        rots += [tile * s, -tile * s]
        s *= 2
    keys = ckks.keygen(P, 42, helpers.galois_elts(P, rots))
    ctx = helpers.gpu_context("ordb")
    helpers.import_keys(ctx, keys)
    helpers.import_encodings(ctx, P, BSZ, kinds=("row0", "col0", "tie"))
    for L in (2, 3):
        D = L * BSZ
        for kind in ("row0s", "rowidx"):
            u = ckks.encode_unscaled(C.mask_slots(kind, BSZ, 1, D, slots=P.slots), P.n)
            ctx.encoding_import(helpers.MASK_IDS[kind], BSZ, 1, D, u)
        ctx.indicator_import(D, C.sinc2_window_coeffs(D))
    yield P, keys, ctx, tiles
    ctx.close()


def test_pair_packed_blocked_circuits_bit_exact(ordb_packed):
    """With the packing keys present the blocked circuits pack their block-pair
    comparisons (and the order statistic's and sort's indicators) 64 to a ciphertext:
    each output block equals the oracle's packed schedule bit for bit and decrypts to
    the noiseless model of the circuit (for ranks also to brute force; the order
    statistic and sort carry the g f comparator's own error at gap 1/8); with
    RK_OPT_PAIR_PACKING = 0 they equal the unpacked schedule."""
    from paper_2412_15126_gb300 import rankfhe
    P, keys, ctx, tiles = ordb_packed
    Bo = C.OracleCkks(P, keys)
    v3 = np.array([0.75, 0.125, 0.5, 0.0, 0.625, 0.25, 0.875, 0.375, 0.3125, 0.5625, 0.1875, 0.9375])
    t3 = np.array([3, 1, 3, 0, 2, 1, 3, 2, 0, 1, 2, 3]) / 8.0
    v2 = np.array([0.75, 0.125, 0.5, 0.0, 0.625, 0.25, 0.875, 0.375])
    cases = [
        (v3, lambda g: ctx.rank_blocked(g), lambda c, p: C.rank_blocked(Bo, c, BSZ, 1, 1, pack=p),
         C.brute_fractional_rank(v3), 0.5),
        (t3, lambda g: ctx.rank_blocked(g, rankfhe.TIES_CORRECT),
         lambda c, p: C.rank_blocked_tc(Bo, c, BSZ, 1, 1, pack=p)[0],
         _plain_blocks(P, t3, lambda Bp, bl: C.rank_blocked_tc(Bp, bl, BSZ, 1, 1)[0]), 1e-3),
        (v2, lambda g: ctx.order_stat_blocked(g, 2), lambda c, p: C.order_statistic_blocked(Bo, c, BSZ, 2, 1, 1, pack=p),
         _plain_blocks(P, v2, lambda Bp, bl: C.order_statistic_blocked(Bp, bl, BSZ, 2, 1, 1)), 1e-3),
        (v2, lambda g: ctx.sort_blocked(g), lambda c, p: C.sort_blocked(Bo, c, BSZ, 1, 1, pack=p),
         _plain_blocks(P, v2, lambda Bp, bl: C.sort_blocked(Bp, bl, BSZ, 1, 1)), 1e-3),
    ]
    for idx, (v, gpu, orc, want, tol) in enumerate(cases):
        cts, g = _encrypt_blocks(P, keys, ctx, v, 80 + 10 * idx)
        ref = orc(cts, tiles)
        got = gpu(g)
        for a, b in zip(got, ref):
            assert a.level == b.level
            assert np.array_equal(a.export(), b.c), idx
        dec = np.concatenate([ctx.decrypt(a) for a in got])
        assert np.max(np.abs(dec - want)) < tol, idx
        ctx.set_option(rankfhe.OPT_PAIR_PACKING, 0)
        try:
            plain = gpu(g)
        finally:
            ctx.set_option(rankfhe.OPT_PAIR_PACKING, 1)
        for a, b in zip(plain, orc(cts, 1)):
            assert np.array_equal(a.export(), b.c), idx


def test_chunked_blocked_circuits_identical(ordb_packed):
    """Stacking budgets of one byte (every step of the blocked circuits in chunks of
    one packing group, every indicator group on its own) leave every output block
    unchanged, bit for bit: rank, tie-corrected rank, order statistic, sort."""
    from paper_2412_15126_gb300 import rankfhe
    P, keys, ctx, tiles = ordb_packed
    v = np.array([0.75, 0.125, 0.5, 0.0, 0.625, 0.25, 0.875, 0.375, 0.3125, 0.5625, 0.1875, 0.9375])
    _, g = _encrypt_blocks(P, keys, ctx, v, 95)
    runs = [lambda: ctx.rank_blocked(g), lambda: ctx.rank_blocked(g, rankfhe.TIES_CORRECT),
            lambda: ctx.order_stat_blocked(g, 5), lambda: ctx.sort_blocked(g)]
    for packing in (1, 0):
        ctx.set_option(rankfhe.OPT_PAIR_PACKING, packing)
        try:
            full = [[b.export() for b in run()] for run in runs]
            ctx.set_option(rankfhe.OPT_STACK_BUDGET, 1)
            ctx.set_option(rankfhe.OPT_INDICATOR_BUDGET, 1)
            small = [[b.export() for b in run()] for run in runs]
        finally:
            ctx.set_option(rankfhe.OPT_STACK_BUDGET, 16 << 30)
            ctx.set_option(rankfhe.OPT_INDICATOR_BUDGET, 4 << 30)
            ctx.set_option(rankfhe.OPT_PAIR_PACKING, 1)
        for a, b in zip(full, small):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
