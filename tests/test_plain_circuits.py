"""Pins for the circuits in the noiseless slot model: the paper's worked examples
(tests/golden/paper_examples.json), brute force over small N and the invariants
of the correctness proofs (Sec. 3.1, Sec. 4, Eq. 3)."""
import numpy as np
import pytest

from oracle import circuits as C


def _mat(B, x, N, q=0):
    return B.values(x)[q * N * N:(q + 1) * N * N].reshape(N, N)


def test_fig1_transc_trace(golden):
    g = golden["fig1_transc_n8"]
    N = 8
    B = C.PlainSlots(N * N, 5)                  # the figure rotates over exactly N^2 slots
    start = np.array(g["start"], dtype=float)
    x = C.PV(start.reshape(-1), 5)
    trace = []
    out = C.trans_c(B, x, N, trace=trace)
    assert [r for r, _ in trace] == g["rotations"]
    for (r, xi), key in zip(trace, ["after_28", "after_14", "after_7"]):
        assert np.array_equal(_mat(B, xi, N), np.array(g[key], dtype=float)), key
    assert np.array_equal(_mat(B, out, N), np.array(g["masked"], dtype=float))


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16])
def test_matrix_ops_brute_force(N):
    slots = 4 * N * N
    B = C.PlainSlots(slots, 10)
    rng = np.random.default_rng(N)
    M = rng.uniform(-1, 1, (N, N))
    X = np.zeros(slots)
    X[: N * N] = M.reshape(-1)
    x = C.PV(X, 10)
    assert np.allclose(_mat(B, C.sum_r(B, x, N), N)[0], M.sum(axis=0))
    assert np.allclose(_mat(B, C.sum_c(B, x, N), N)[:, 0], M.sum(axis=1))
    row = np.zeros(slots)
    row[:N] = M[0]
    col = np.zeros(slots)
    col[: N * N: N] = M[:, 0]
    assert np.allclose(_mat(B, C.repl_r(B, C.PV(row, 10), N), N), np.tile(M[0], (N, 1)))
    assert np.allclose(_mat(B, C.repl_c(B, C.PV(col, 10), N), N), np.tile(M[:, 0][:, None], (1, N)))
    tr = _mat(B, C.trans_r(B, C.PV(row, 10), N), N)
    expect = np.zeros((N, N))
    expect[:, 0] = M[0]
    assert np.allclose(tr, expect)
    tc = _mat(B, C.trans_c(B, C.PV(col, 10), N), N)
    expect = np.zeros((N, N))
    expect[0] = M[:, 0]
    assert np.allclose(tc, expect)


def test_fig2_rank_example(golden):
    g = golden["fig2_rank"]
    v = np.array(g["input"]) / 64.0
    B = C.PlainSlots(64, 40)
    Cm = C.comparison_matrix(B, B.fresh(v), 4, 3, 2)
    assert np.max(np.abs(_mat(B, Cm, 4) - np.array(g["C"]))) < 1e-6
    assert np.all(_mat(B, Cm, 4)[np.eye(4, dtype=bool)] == 0.5)       # Cmp(x, x) = 1/2 exactly
    S = C.sum_r(B, Cm, 4)
    assert np.max(np.abs(B.values(S)[:4] - np.array(g["sumR"]))) < 1e-5
    B2 = C.PlainSlots(64, 40)
    R = C.rank(B2, B2.fresh(v), 4, 3, 2)
    assert np.max(np.abs(B2.values(R)[:4] - np.array(g["rank"]))) < 1e-5


def test_sec31_fractional_padded(golden):
    g = golden["sec31_fractional"]
    v = np.array(g["input"]) / 64.0
    B = C.PlainSlots(256, 40)
    R = C.rank(B, B.fresh(np.r_[v, np.zeros(3)]), 8, 3, 2, n_real=5)
    assert np.max(np.abs(B.values(R)[:5] - np.array(g["rank"]))) < 1e-5
    assert np.allclose(C.brute_fractional_rank(g["input"]), g["rank"])


def test_fig4_tie_offset(golden):
    g = golden["fig4_tie_offset"]
    v = np.array(g["input"]) / 64.0
    B = C.PlainSlots(64, 40)
    Cm = C.comparison_matrix(B, B.fresh(v), 4, 3, 2)
    E, U, T, F = C.tie_offset_unfolded(B, Cm, 4)
    assert np.max(np.abs(_mat(B, E, 4) - np.array(g["E"]))) < 1e-5
    assert np.max(np.abs(B.values(U)[:4] - np.array(g["U"]))) < 1e-5
    assert np.max(np.abs(B.values(T)[:4] - np.array(g["T"]))) < 1e-5
    assert np.max(np.abs(B.values(F)[:4] - np.array(g["F"]))) < 1e-5
    B2 = C.PlainSlots(64, 40)
    R = C.rank_tie_corrected(B2, B2.fresh(v), 4, 3, 2)
    assert np.max(np.abs(B2.values(R)[:4] - np.array(g["corrected_rank"]))) < 1e-5
    assert np.allclose(C.brute_tie_corrected_rank(g["input"]), g["corrected_rank"])


def test_rotation_count_rank(golden):
    # Sec. 3.1: 4 ceil(log N) rotations for ranking; 28 at N = 128 (Sec. 6 argmin count).
    for N in (2, 8, 32, 128):
        B = C.PlainSlots(max(2 * N * N, 64), 40, radix2=True)   # one doubling a step, as printed
        C.rank(B, B.fresh(np.linspace(0, 0.9, N)), N, 4, 2)
        assert B.counts["rot"] == 4 * int(np.log2(N))
    assert golden["argmin_counts"]["rotations"] == 4 * 7


@pytest.mark.parametrize("seed", range(6))
def test_rank_brute_force_and_invariants(seed):
    rng = np.random.default_rng(seed)
    N = [4, 8, 16, 32, 64, 128][seed]
    gap = 2.0 ** -9
    v = np.sort(rng.uniform(0, 1 - (N - 1) * gap, N)) + np.arange(N) * gap
    v = rng.permutation(v)
    B = C.PlainSlots(max(2 * N * N, 64), 40)
    R = B.values(C.rank(B, B.fresh(v), N, 4, 2))[:N]
    assert np.max(np.abs(R - C.brute_fractional_rank(v))) < 0.25
    assert abs(R.sum() - N * (N + 1) / 2) < 0.25


@pytest.mark.parametrize("seed", range(4))
def test_tie_corrected_is_permutation(seed):
    rng = np.random.default_rng(100 + seed)
    N = [8, 16, 32, 64][seed]
    v = rng.integers(0, 64, N) / 64.0
    B = C.PlainSlots(max(2 * N * N, 64), 40)
    R = B.values(C.rank_tie_corrected(B, B.fresh(v), N, 3, 2))[:N]
    k = C.brute_tie_corrected_rank(v)
    assert np.max(np.abs(R - k)) < 0.25
    assert sorted(np.rint(R).astype(int)) == list(range(1, N + 1))
    # v_j is the k_j-th order statistic (Sec. 4, proof point 2)
    s = np.sort(v)
    assert all(s[int(kj) - 1] == vj for kj, vj in zip(np.rint(R), v))


def test_block_complement_identity():
    # Eq. 3: C_{i,j} = (1 - C_{j,i})^T for blocks of a longer vector
    rng = np.random.default_rng(7)
    Bsz = 8
    vi = rng.uniform(0, 1, Bsz)
    vj = rng.uniform(0, 1, Bsz)

    def block_cmp(a, b):
        B = C.PlainSlots(2 * Bsz * Bsz, 40)
        VR = C.repl_r(B, B.fresh(a), Bsz)
        VC = C.repl_c(B, C.trans_r(B, B.fresh(b), Bsz), Bsz)
        X = B.sub(B.level_down(VR, B.level(VC)), VC)
        return _mat(B, C.cmp(B, X, 4, 2), Bsz)

    Cij = block_cmp(vi, vj)
    Cji = block_cmp(vj, vi)
    assert np.max(np.abs(Cij - (1 - Cji).T)) < 1e-5


def test_packed_queries_do_not_leak():
    # Q queries packed at stride N^2: each query's ranks equal its own brute force.
    N, Q = 8, 4
    rng = np.random.default_rng(11)
    vs = [rng.permutation(np.linspace(0.05, 0.95, N)) for _ in range(Q)]
    slots = Q * N * N * 2
    B = C.PlainSlots(slots, 40)
    X = np.zeros(slots)
    for q, v in enumerate(vs):
        X[q * N * N: q * N * N + N] = v
    R = B.values(C.rank(B, C.PV(X, 40), N, 4, 2, Q=Q))
    for q, v in enumerate(vs):
        assert np.max(np.abs(R[q * N * N: q * N * N + N] - C.brute_fractional_rank(v))) < 1e-3


@pytest.mark.parametrize("Bsz,L", [(4, 2), (4, 3), (8, 4), (64, 2)])
def test_blocked_rank_equals_whole_vector_rank(Bsz, L):
    """Alg. 7 on L blocks gives the ranks of the whole vector (for Bsz = 64, L = 2 the
    single-ciphertext N = 128 ranks)."""
    rng = np.random.default_rng(Bsz * 10 + L)
    N = Bsz * L
    v = rng.permutation(np.linspace(0.01, 0.98, N))
    slots = max(2 * Bsz * Bsz, 64)
    B = C.PlainSlots(slots, 40)
    Rs = C.rank_blocked(B, [B.fresh(v[i * Bsz:(i + 1) * Bsz]) for i in range(L)], Bsz, 4, 2)
    got = np.concatenate([B.values(R)[:Bsz] for R in Rs])
    assert np.max(np.abs(got - C.brute_fractional_rank(v))) < 1e-3
    assert len({R.level for R in Rs}) == 1 and Rs[0].level == 40 - 3 - 3 * 6
    if N <= 128 and N & (N - 1) == 0:
        B1 = C.PlainSlots(2 * N * N, 40)
        single = B1.values(C.rank(B1, B1.fresh(v), N, 4, 2))[:N]
        assert np.max(np.abs(got - single)) < 1e-3


def test_blocked_rank_two_packed_queries():
    """Two blocked queries packed at stride Bsz^2 in the same block ciphertexts keep
    their own ranks (Q = 2, as the batched form packs N = 512 queries)."""
    Bsz, L, Q = 8, 3, 2
    rng = np.random.default_rng(5)
    vs = [rng.permutation(np.linspace(0.02, 0.97, Bsz * L)) for _ in range(Q)]
    slots = Q * Bsz * Bsz * 2
    B = C.PlainSlots(slots, 40)
    blocks = []
    for i in range(L):
        x = np.zeros(slots)
        for q in range(Q):
            x[q * Bsz * Bsz: q * Bsz * Bsz + Bsz] = vs[q][i * Bsz:(i + 1) * Bsz]
        blocks.append(C.PV(x, 40))
    Rs = C.rank_blocked(B, blocks, Bsz, 4, 2, Q=Q)
    for q in range(Q):
        got = np.concatenate([B.values(R)[q * Bsz * Bsz: q * Bsz * Bsz + Bsz] for R in Rs])
        assert np.max(np.abs(got - C.brute_fractional_rank(vs[q]))) < 1e-3


def test_fig3_sort_example(golden):
    g = golden["fig3_sort"]
    v = np.array(g["input"]) / 64.0
    B = C.PlainSlots(64, 40)
    S = B.values(C.sort(B, B.fresh(v), 4, 3, 2))
    assert np.max(np.abs(S[:4] - np.array(g["sorted"]) / 64.0)) < 1e-4
    assert np.all(np.abs(S[4:16]) < 1e-9)


def test_cheb_ps_matches_chebyshev_sum():
    """The recursive split p = q T_m + r reproduces sum_i c_i T_i(t) (numpy's chebval)."""
    rng = np.random.default_rng(3)
    for length in (4, 8, 16, 64, 256):
        c = rng.uniform(-1, 1, length)
        t = np.linspace(-1, 1, 97)
        B = C.PlainSlots(97, 40)
        got = B.values(C.cheb_ps(B, C.PV(t.copy(), 40), c))
        assert np.max(np.abs(got - np.polynomial.chebyshev.chebval(t, c))) < 1e-9
        assert B.level is not None


def test_cheb_ps_depth():
    for length in (8, 64, 1024):
        B = C.PlainSlots(4, 40)
        out = C.cheb_ps(B, C.PV(np.zeros(4), 40), np.ones(length))
        assert out.level == 40 - C.cheb_depth(length)


@pytest.mark.parametrize("N", [4, 8, 32, 128])
def test_sinc2_window_is_indicator_at_integers(N):
    c = C.sinc2_window_coeffs(N)
    assert len(c) == max(8 * N, 128)
    ks = np.arange(-N + 1, N)
    vals = np.polynomial.chebyshev.chebval(ks / N, c)
    assert np.max(np.abs(vals - (ks == 0))) < 1e-9


@pytest.mark.parametrize("seed", range(4))
def test_order_statistics_and_sort_brute_force(seed):
    rng = np.random.default_rng(200 + seed)
    N = [8, 16, 32, 64][seed]
    v = rng.integers(0, 16, N) / 16.0
    s = np.sort(v)
    for k in (1, N // 2, N):
        B = C.PlainSlots(max(2 * N * N, 64), 40)
        O = B.values(C.order_statistic(B, B.fresh(v), N, k, 3, 2))[:N]
        first = np.zeros(N)
        first[int(np.where(C.brute_tie_corrected_rank(v) == k)[0][0])] = 1
        assert np.max(np.abs(O - first)) < 1e-6
    B = C.PlainSlots(max(2 * N * N, 64), 40)
    O = B.values(C.order_statistic(B, B.fresh(v), N, 1, 3, 2, ties="all"))[:N]
    assert np.max(np.abs(O - (v == v.min()))) < 1e-6
    B = C.PlainSlots(max(2 * N * N, 64), 40)
    O = B.values(C.order_statistic(B, B.fresh(v), N, N, 3, 2, ties="all"))[:N]
    assert np.max(np.abs(O - (v == v.max()))) < 1e-6
    B = C.PlainSlots(max(2 * N * N, 64), 40)
    S = B.values(C.sort(B, B.fresh(v), N, 3, 2))[:N]
    assert np.max(np.abs(S - s)) < 1e-6


def _blocks(B, v, Bsz):
    return [B.fresh(v[i * Bsz:(i + 1) * Bsz]) for i in range(len(v) // Bsz)]


@pytest.mark.parametrize("Bsz,L", [(4, 2), (4, 3), (8, 2), (2, 4)])
def test_blocked_tie_corrected_rank_is_the_stable_rank(Bsz, L):
    """Alg. 7 with Alg. 6 over blocks: the global stable rank (equal values ordered by
    block, then position), also when divided by the total length."""
    rng = np.random.default_rng(100 + Bsz * L)
    N = Bsz * L
    v = rng.integers(0, max(N // 2, 2), N) / (2.0 * N)      # ties across and within blocks
    B = C.PlainSlots(max(2 * Bsz * Bsz, 64), 60)
    Rs, _ = C.rank_blocked_tc(B, _blocks(B, v, Bsz), Bsz, 4, 2)
    got = np.concatenate([B.values(R)[:Bsz] for R in Rs])
    assert np.max(np.abs(got - C.brute_tie_corrected_rank(v))) < 1e-3
    assert len({R.level for R in Rs}) == 1 and Rs[0].level == 60 - 1 - 18 - 3
    Bs = C.PlainSlots(max(2 * Bsz * Bsz, 64), 60)
    Rs2, _ = C.rank_blocked_tc(Bs, _blocks(Bs, v, Bsz), Bsz, 4, 2, scaled=True)
    got2 = np.concatenate([Bs.values(R)[:Bsz] for R in Rs2])
    assert np.max(np.abs(got2 * N - C.brute_tie_corrected_rank(v))) < 1e-3


def test_blocked_tie_corrected_rank_one_block_is_alg6():
    """With one block the blocked schedule is the single-ciphertext fold of Alg. 6."""
    v = np.array([3, 1, 3, 0, 2, 1, 3, 2]) / 8.0
    B = C.PlainSlots(128, 60)
    Rs, _ = C.rank_blocked_tc(B, [B.fresh(v)], 8, 4, 2)
    ref = C.rank_tie_corrected(B, B.fresh(v), 8, 4, 2)
    assert np.array_equal(B.values(Rs[0]), B.values(ref))


@pytest.mark.parametrize("k", [1, 5, 12])
def test_blocked_order_statistic_one_hot(k):
    """Alg. 4 on blocked tie-corrected ranks: one 1 at the first element of rank k."""
    Bsz, L = 4, 3
    v = np.array([5, 2, 9, 2, 7, 0, 5, 11, 0, 3, 9, 6]) / 24.0
    B = C.PlainSlots(64, 60)
    Os = C.order_statistic_blocked(B, _blocks(B, v, Bsz), Bsz, k, 4, 2)
    got = np.concatenate([B.values(O)[:Bsz] for O in Os])
    want = (C.brute_tie_corrected_rank(v) == k).astype(float)
    assert want.sum() == 1
    assert np.max(np.abs(got - want)) < 1e-3


@pytest.mark.parametrize("Bsz,L", [(4, 3), (2, 4), (8, 2)])
def test_blocked_sort_is_sorted_vector(Bsz, L):
    """Alg. 8 on tie-corrected ranks returns the sorted vector block by block (ties kept)."""
    rng = np.random.default_rng(7 + Bsz * L)
    N = Bsz * L
    v = rng.integers(0, N, N) / (2.0 * N)
    B = C.PlainSlots(max(2 * Bsz * Bsz, 64), 80)
    Ss = C.sort_blocked(B, _blocks(B, v, Bsz), Bsz, 4, 2)
    got = np.concatenate([B.values(S)[:Bsz] for S in Ss])
    assert np.max(np.abs(got - np.sort(v))) < 1e-3
    for S in Ss:   # nothing outside row 0 of each block
        assert np.all(np.abs(B.values(S)[Bsz:Bsz * Bsz]) < 1e-6)


@pytest.mark.parametrize("name", ["ties", "distinct"])
def test_order_value_and_median(name):
    """Value retrieval SumC(O . V) (Sec. 3.2) gives the k-th smallest value; the median
    is the mean of the two middle statistics for even N (numpy's median)."""
    v = {"ties": np.array([3, 1, 3, 0, 2, 1, 3, 2]) / 8.0,
         "distinct": np.array([0.5, 0.125, 0.875, 0.25, 0.0, 0.625, 0.375, 0.75])}[name]
    for k in (1, 4, 5, 8):
        B = C.PlainSlots(128, 60)
        got = B.values(C.order_value(B, B.fresh(v), 8, k, 4, 2))
        assert abs(got[0] - np.sort(v)[k - 1]) < 1e-6
    B = C.PlainSlots(128, 60)
    got = B.values(C.median(B, B.fresh(v), 8, 4, 2))
    assert abs(got[0] - np.median(v)) < 1e-6
    assert np.all(np.abs(got[1:8]) < 1e-6)          # row 0 keeps only column 0 (SumC's mask)


def test_order_value_middle_statistic():
    """The value of a middle statistic (the odd-N median's form) of distinct values."""
    v = np.array([0.3, 0.9, 0.1, 0.6, 0.2, 0.8, 0.4, 0.7])
    B = C.PlainSlots(128, 60)
    got = B.values(C.order_value(B, B.fresh(v), 8, 4, 4, 2))
    assert abs(got[0] - np.sort(v)[3]) < 1e-6


def test_chebyshev_comparator_closed_form_and_ties():
    """The Chebyshev comparator evaluated by Paterson-Stockmeyer equals numpy's chebval
    of its coefficients, is 1/2 exactly at x = 0, and tends to the step away from 0."""
    for count in (16, 64, 256):
        cc = C.ChebCmp(count)
        x = np.linspace(-1, 1, 401)
        B = C.PlainSlots(401, 40)
        got = B.values(C.cmp(B, C.PV(x.copy(), 40), cc, 0))
        assert np.max(np.abs(got - np.polynomial.chebyshev.chebval(x, cc.coeffs))) < 1e-9
        assert got[200] == 0.5
        far = np.abs(x) > 8.0 / count
        assert np.max(np.abs(got[far] - (x[far] > 0))) < 0.1


def test_chebyshev_comparator_reproduces_fig6(golden):
    """Rank error against comparison depth with the Chebyshev comparator (App. B,
    Fig. 6): on seeded uniform 128-element vectors the mean error of the ranks lies
    within 25 % of the paper's printed average at every depth 6..13."""
    g = golden["fig6_rank_error"]
    rng = np.random.default_rng(66)
    vs = [rng.uniform(0, 1, 128) for _ in range(8)]
    for depth, paper in zip(g["depth"], g["avg_error"]):
        if depth > 13:
            continue
        cc = C.ChebCmp(1 << (depth - 1))
        errs = []
        for v in vs:
            B = C.PlainSlots(2 * 128 * 128, 40)
            R = B.values(C.rank(B, B.fresh(v), 128, cc, 0))[:128]
            errs.append(np.abs(R - C.brute_fractional_rank(v)))
        mean = float(np.mean(errs))
        assert abs(mean - paper) < 0.25 * paper, (depth, mean, paper)
