"""The encrypted oracle runs the circuits end to end on the n = 2^13 parameter set
(14 primes of ~40 bits plus one special prime) and decrypts to the brute-force
ranks; its decrypted comparison matrix matches the noiseless slot model."""
import numpy as np
import pytest

from oracle import ckks, circuits as C
from paper_2412_15126_gb300 import inputs


def rotation_set(N):
    k = int(np.log2(N))
    rs = set()
    for i in range(k):
        rs.update({-(N << i), N << i, -(1 << i), 1 << i})
    for i in range(1, k + 1):
        rs.update({-((N * (N - 1)) >> i), (N * (N - 1)) >> i})
    return rs


@pytest.fixture(scope="module")
def small():
    P = ckks.gen_params(13, 14, 40, 40, 1, 61, 1)
    gal = [ckks.galois_left(r % P.slots, P.n) for r in rotation_set(8)]
    keys = ckks.keygen(P, 2024, gal)
    return P, keys


@pytest.mark.parametrize("seed", [1, 2])
def test_encrypted_rank_n8(small, seed):
    P, keys = small
    v = inputs.gap_vector(8, 0.05, seed)
    ct = ckks.encrypt(P, keys, v, seed)
    B = C.OracleCkks(P, keys)
    R = C.rank(B, ct, 8, 2, 1)
    got = B.values(R)[:8]
    assert np.max(np.abs(got - C.brute_fractional_rank(v))) < 0.25
    # the same schedule in the noiseless model, slot by slot
    Bp = C.PlainSlots(P.slots, P.L)
    ideal = Bp.values(C.rank(Bp, Bp.fresh(v), 8, 2, 1))
    assert R.level == Bp.top - 11
    assert np.max(np.abs(B.values(R) - ideal)) < 2.0 ** -12


def test_rank_out_level_and_trimmed_rank(small):
    """With q_0 of 40 bits at scale 2^40, level 0 cannot hold ranks up to 8, so the
    result keeps level 1 (a 60-bit q_0 at 2^45 holds ranks up to 2^13 at level 0); the
    trimmed schedule decrypts to the brute-force ranks from level 1, and without
    trimming the same levels are simply not spent."""
    P, keys = small
    assert C.rank_out_level(P, 8) == 1
    P60 = ckks.gen_params(10, 6, 60, 45, 1, 61, 1)
    assert C.rank_out_level(P60, 128) == 0 and C.rank_out_level(P60, 1 << 14) == 1
    v = inputs.gap_vector(8, 0.05, 21)
    ct = ckks.encrypt(P, keys, v, 21)
    B = C.OracleCkks(P, keys)
    R = C.rank(B, ct, 8, 2, 1, trim=True)
    assert R.level == 1
    assert np.max(np.abs(B.values(R)[:8] - C.brute_fractional_rank(v))) < 0.25


def test_encrypted_tie_corrected_rank(small):
    P, keys = small
    v = np.array([3, 1, 3, 0, 2, 1, 3, 2]) / 4.0
    ct = ckks.encrypt(P, keys, v, 5)
    B = C.OracleCkks(P, keys)
    R = C.rank_tie_corrected(B, ct, 8, 2, 1)
    got = B.values(R)[:8]
    assert np.max(np.abs(got - C.brute_tie_corrected_rank(v))) < 0.25


@pytest.fixture(scope="module")
def deep():
    P = ckks.gen_params(11, 24, 60, 40, 2, 61, 2)
    gal = [ckks.galois_left(r % P.slots, P.n) for r in rotation_set(8)]
    return P, ckks.keygen(P, 7, gal)


def test_encrypted_argmin_argmax_sort_n8(deep):
    P, keys = deep
    v = np.array([3, 1, 3, 0, 2, 1, 3, 2]) / 4.0
    ct = ckks.encrypt(P, keys, v, 2)
    B = C.OracleCkks(P, keys)
    o = B.values(C.order_statistic(B, ct, 8, 1, 2, 1))[:8]
    assert np.max(np.abs(o - (np.arange(8) == 3))) < 0.01
    o = B.values(C.order_statistic(B, ct, 8, 8, 2, 1, ties="all"))[:8]
    assert np.max(np.abs(o - (v == v.max()))) < 0.01
    s = B.values(C.sort(B, ct, 8, 2, 1))[:8]
    assert np.max(np.abs(s - np.sort(v))) < 0.01
