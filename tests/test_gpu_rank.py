"""GPU parity of the ranking circuits (Alg. 3, Alg. 6 folded).

* n = 2^13 set, N = 8: with the oracle's keys, input ciphertext and mask
  encodings imported, the CUDA rank circuit returns the oracle's ciphertext bit
  for bit (plain and tie-corrected).
* n = 2^16, 28 limbs (the 128-element workload) in the launch configuration the
  benchmark times: one rotation and one product checked bit for bit against the
  oracle on imported keys; the full circuit on the library's own keys decrypts to
  the brute-force ranks within 0.25 and to the noiseless slot model.
"""
import numpy as np
import pytest

from oracle import ckks, circuits as C
from paper_2412_15126_gb300 import inputs
from tests import helpers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg1():
    P = helpers.oracle_params("cfg1")
    keys = ckks.keygen(P, 2024, helpers.galois_elts(P, helpers.rotation_set(8)))
    ctx = helpers.gpu_context("cfg1")
    helpers.import_keys(ctx, keys)
    helpers.import_encodings(ctx, P, 8)
    yield P, keys, ctx
    ctx.close()


def test_compare_matrix_n8_bit_exact(cfg1):
    P, keys, ctx = cfg1
    v = inputs.gap_vector(8, 0.05, 4)
    ct = ckks.encrypt(P, keys, v, 4)
    Cm = C.comparison_matrix(C.OracleCkks(P, keys), ct, 8, 2, 1)
    g = ctx.compare_matrix(ctx.ct_import(ct.c, ct.level, N=8))
    assert np.array_equal(g.export(), Cm.c)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rank_n8_bit_exact(cfg1, seed):
    P, keys, ctx = cfg1
    v = inputs.gap_vector(8, 0.05, seed)
    ct = ckks.encrypt(P, keys, v, seed)
    B = C.OracleCkks(P, keys)
    R = C.rank(B, ct, 8, 2, 1)
    g = ctx.rank(ctx.ct_import(ct.c, ct.level, N=8))
    assert g.level == R.level
    assert np.array_equal(g.export(), R.c)
    got = ctx.decrypt(g)
    assert np.max(np.abs(got - C.brute_fractional_rank(v))) < 0.25


def test_rank_tie_corrected_n8_bit_exact(cfg1):
    P, keys, ctx = cfg1
    v = np.array([3, 1, 3, 0, 2, 1, 3, 2]) / 4.0
    ct = ckks.encrypt(P, keys, v, 9)
    B = C.OracleCkks(P, keys)
    R = C.rank_tie_corrected(B, ct, 8, 2, 1)
    g = ctx.rank(ctx.ct_import(ct.c, ct.level, N=8), flags=1)
    assert np.array_equal(g.export(), R.c)
    assert np.max(np.abs(ctx.decrypt(g) - C.brute_tie_corrected_rank(v))) < 0.25


def test_rank_padded_n5(cfg1):
    P, keys, ctx = cfg1
    helpers.import_encodings(ctx, P, 8, n_real=5, kinds=())
    v = inputs.gap_vector(5, 0.05, 11)
    ct = ckks.encrypt(P, keys, np.r_[v, np.zeros(3)], 11)
    B = C.OracleCkks(P, keys)
    R = C.rank(B, ct, 8, 2, 1, n_real=5)
    g = ctx.rank(ctx.ct_import(ct.c, ct.level, N=8, n_real=5))
    assert np.array_equal(g.export(), R.c)
    assert np.max(np.abs(ctx.decrypt(g) - C.brute_fractional_rank(v))) < 0.25


@pytest.mark.parametrize("N, n_real", [(1, 1), (2, 2), (2, 1)])
def test_rank_degenerate_lengths(cfg1, N, n_real):
    """The degenerate lengths: one element (no rotation at all: rank 1), two, and one
    real value padded to two; bit-exact with the oracle."""
    P, keys, ctx = cfg1
    helpers.import_encodings(ctx, P, N)
    if n_real != N:
        helpers.import_encodings(ctx, P, N, n_real=n_real, kinds=())
    v = inputs.gap_vector(n_real, 0.05, 40 + N + n_real)
    ct = ckks.encrypt(P, keys, np.r_[v, np.zeros(N - n_real)], 17)
    R = C.rank(C.OracleCkks(P, keys), ct, N, 2, 1, n_real=n_real)
    g = ctx.rank(ctx.ct_import(ct.c, ct.level, N=N, n_real=n_real))
    assert np.array_equal(g.export(), R.c)
    assert np.max(np.abs(ctx.decrypt(g)[:n_real] - C.brute_fractional_rank(v))) < 0.25


def test_rank_rejects_empty_and_bad_lengths(cfg1):
    """No real value, a length that is not a power of two, or N^2 beyond the slots:
    RK_EINVAL before any kernel runs."""
    from paper_2412_15126_gb300 import rankfhe
    P, keys, ctx = cfg1
    ct = ckks.encrypt(P, keys, np.zeros(8), 3)
    for kw in (dict(N=8, n_real=0), dict(N=6), dict(N=1 << 12)):
        with pytest.raises(rankfhe.RkError) as e:
            ctx.rank(ctx.ct_import(ct.c, ct.level, **kw))
        assert e.value.status == rankfhe.RK_EINVAL


def test_rank_trimmed_levels_bit_exact(cfg1):
    """RK_OPT_TRIM_LEVELS: the input is brought down to the lowest level the rank
    needs (keeping one more level when q_0 cannot hold ranks at the scale); the
    result equals the oracle's trimmed schedule bit for bit."""
    from paper_2412_15126_gb300 import rankfhe
    P, keys, ctx = cfg1
    v = inputs.gap_vector(8, 0.05, 12)
    ct = ckks.encrypt(P, keys, v, 12)
    R = C.rank(C.OracleCkks(P, keys), ct, 8, 2, 1, trim=True)
    ctx.set_option(rankfhe.OPT_TRIM_LEVELS, 1)
    try:
        g = ctx.rank(ctx.ct_import(ct.c, ct.level, N=8))
    finally:
        ctx.set_option(rankfhe.OPT_TRIM_LEVELS, 0)
    assert g.level == R.level == C.rank_out_level(P, 8)
    assert np.array_equal(g.export(), R.c)
    assert np.max(np.abs(ctx.decrypt(g) - C.brute_fractional_rank(v))) < 0.25


def test_depth_error(cfg1):
    from paper_2412_15126_gb300 import rankfhe
    P, keys, ctx = cfg1
    ct = ckks.encrypt(P, keys, np.linspace(0, 0.9, 8), 3, level=5)
    with pytest.raises(rankfhe.RkError) as e:
        ctx.rank(ctx.ct_import(ct.c, ct.level, N=8))
    assert e.value.status == rankfhe.RK_EDEPTH


def test_cfg2_single_ops_bit_exact():
    P = helpers.oracle_params("cfg2")
    r = -128
    keys = ckks.keygen(P, 5, helpers.galois_elts(P, [r]))
    ctx = helpers.gpu_context("cfg2")
    helpers.import_keys(ctx, keys)
    v = inputs.gap_vector(128, 2.0 ** -9, 1)
    ct = ckks.encrypt(P, keys, v, 1)
    g = ctx.ct_import(ct.c, ct.level, N=128)
    assert np.array_equal(ctx.rotate(g, r).export(), ckks.rotate(P, keys, ct, r).c)
    assert np.array_equal(ctx.mul(g, g).export(), ckks.mul(P, keys, ct, ct).c)
    ctx.close()


@pytest.fixture(scope="module")
def cfg2_gpu_keys():
    ctx = helpers.gpu_context("cfg2")
    ctx.keygen(2025, 128)
    yield ctx
    ctx.close()


@pytest.mark.parametrize("seed", [1, 2])
def test_cfg2_rank_n128_decrypts_to_ranks(cfg2_gpu_keys, seed):
    ctx = cfg2_gpu_keys
    v = inputs.gap_vector(128, 2.0 ** -9, seed)
    g = ctx.rank(ctx.encrypt(v, N=128))
    got = ctx.decrypt(g)
    assert np.max(np.abs(got - C.brute_fractional_rank(v))) < 0.25
    # the full slot vector against the noiseless model of the same schedule
    P = helpers.oracle_params("cfg2")
    Bp = C.PlainSlots(P.slots, P.L)
    ideal = Bp.values(C.rank(Bp, Bp.fresh(v), 128, 4, 2))
    assert g.level == P.L - 20
    assert np.max(np.abs(ctx.decrypt_slots(g) - ideal)) < 2.0 ** -6


def test_cfg2_comparison_matrix_slots(cfg2_gpu_keys):
    """Comparison-matrix slots within 2^-10 of Cmp (Eq. 1) for every pair outside the
    input gap, and of the noiseless model everywhere."""
    ctx = cfg2_gpu_keys
    N = 128
    v = inputs.gap_vector(N, 2.0 ** -9, 7)
    Cm = ctx.compare_matrix(ctx.encrypt(v, N=N))
    got = ctx.decrypt_slots(Cm)[: N * N].reshape(N, N)
    i, j = np.indices((N, N))
    exact = np.where(v[j] > v[i], 1.0, np.where(v[j] < v[i], 0.0, 0.5))
    assert np.max(np.abs(got - exact)) < 2.0 ** -10
    P = helpers.oracle_params("cfg2")
    Bp = C.PlainSlots(P.slots, P.L)
    ideal = Bp.values(C.comparison_matrix(Bp, Bp.fresh(v), N, 4, 2))
    assert np.max(np.abs(ctx.decrypt_slots(Cm) - ideal)) < 2.0 ** -10


def test_cfg2_trimmed_rank_n128(cfg2_gpu_keys):
    """The 128-element rank with RK_OPT_TRIM_LEVELS: it leaves at level 0 and still
    decrypts to the brute-force ranks within 0.25."""
    from paper_2412_15126_gb300 import rankfhe
    ctx = cfg2_gpu_keys
    v = inputs.gap_vector(128, 2.0 ** -9, 77)
    ctx.set_option(rankfhe.OPT_TRIM_LEVELS, 1)
    try:
        g = ctx.rank(ctx.encrypt(v, N=128))
    finally:
        ctx.set_option(rankfhe.OPT_TRIM_LEVELS, 0)
    assert g.level == 0
    assert np.max(np.abs(ctx.decrypt(g) - C.brute_fractional_rank(v))) < 0.25


def test_cfg2_rank_n16_and_n64(cfg2_gpu_keys):
    ctx = cfg2_gpu_keys
    for N in (16, 64):
        v = inputs.gap_vector(N, 2.0 ** -9, N)
        got = ctx.decrypt(ctx.rank(ctx.encrypt(v, N=N)))
        assert np.max(np.abs(got - C.brute_fractional_rank(v))) < 0.25


def test_cfg3_tie_corrected_n128():
    ctx = helpers.gpu_context("cfg3")
    ctx.keygen(2026, 128)
    v = inputs.grid_vector(128, 64, 1)
    got = ctx.decrypt(ctx.rank(ctx.encrypt(v, N=128), flags=1))
    k = C.brute_tie_corrected_rank(v)
    assert np.max(np.abs(got - k)) < 0.25
    assert sorted(np.rint(got).astype(int)) == list(range(1, 129))
    ctx.close()
