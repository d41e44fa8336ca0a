"""Pins of the doubling chains taken two steps at a time (x + (x << a) + (x << b) +
(x << a + b), one ModDown for the three rotations) against the chains of the paper's
algorithms one step at a time (Alg. 1, 2, 8-11).

* Noiseless slot model: every chain and every circuit gives the same slot values
  either way (rotations compose additively).
* RNS-CKKS: rotate_sum decrypts to x + sum of the shifted slot vectors; it differs
  from adding the separate rotations only by the ModDown's rounding (a few units per
  coefficient); ranks over chains of pairs decrypt to the brute-force ranks.
"""
import math

import numpy as np
import pytest

from oracle import ckks, circuits as C
from paper_2412_15126_gb300 import inputs
from tests import helpers


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 128])
def test_chains_of_pairs_equal_single_steps(N):
    slots = max(2 * N * N, 64)
    rng = np.random.default_rng(N)
    x = rng.uniform(-1, 1, slots)
    for amounts in (C.repl_r_amounts(N), C.trans_r_amounts(N), [1 << i for i in range(int(math.log2(N)))],
                    [-(1 << i) for i in range(int(math.log2(N)))]):
        B4, B2 = C.PlainSlots(slots, 5), C.PlainSlots(slots, 5, radix2=True)
        a = B4.values(C.chain(B4, B4.fresh(x), amounts))
        b = B2.values(C.chain(B2, B2.fresh(x), amounts))
        assert np.max(np.abs(a - b)) < 1e-12
        steps = C.chain_pairs(B4, amounts)
        assert sum(C.steps_taken(st) for st in steps) == len(amounts)
        assert len(steps) == (len(amounts) + 1) // 2


@pytest.mark.parametrize("N", [4, 8, 32])
def test_circuits_over_pairs_equal_single_steps(N):
    """rank, tie-corrected rank, order statistic and sort: the same row values."""
    v = inputs.grid_vector(N, max(N // 2, 2), 3 * N)
    slots = max(2 * N * N, 64)
    runs = [
        lambda B: C.rank(B, B.fresh(v), N, 2, 1),
        lambda B: C.rank_tie_corrected(B, B.fresh(v), N, 2, 1),
        lambda B: C.order_statistic(B, B.fresh(v), N, 1, 2, 1),
        lambda B: C.sort(B, B.fresh(v), N, 2, 1),
    ]
    for run in runs:
        B4, B2 = C.PlainSlots(slots, 60), C.PlainSlots(slots, 60, radix2=True)
        a, b = run(B4), run(B2)
        assert a.level == b.level
        assert np.max(np.abs(B4.values(a) - B2.values(b))) < 1e-9
        assert B4.counts["mul"] == B2.counts["mul"]


@pytest.fixture(scope="module")
def small():
    P = ckks.gen_params(10, 6, 60, 40, 2, 61, 2)
    rs = [3, 5, 8, 7, 13]
    keys = ckks.keygen(P, 71, [ckks.galois_left(r, P.n) for r in rs])
    z = np.random.default_rng(72).uniform(-1, 1, P.slots)
    return P, keys, z, ckks.encrypt(P, keys, z, 73)


def test_rotate_sum_decrypts_to_the_sum_of_shifts(small):
    P, keys, z, ct = small
    out = ckks.rotate_sum(P, keys, ct, [3, 5, 8])
    want = z + np.roll(z, -3) + np.roll(z, -5) + np.roll(z, -8)
    assert np.max(np.abs(ckks.decrypt(P, keys, out) - want)) < 2.0 ** -20
    assert out.level == ct.level


def test_rotate_sum_differs_from_added_rotations_by_rounding_only(small):
    """The ModDown of the summed inner products against three ModDowns: the
    ciphertexts differ by at most 3 units a coefficient (each ModDown is round(u / P)
    up to its centred conversion's error, so the sum of three differs from one of the
    sum by the rounding of three terms), and both decrypt alike."""
    P, keys, z, ct = small
    one = ckks.rotate_sum(P, keys, ct, [3, 5, 8])
    sep = ct
    for r in (3, 5, 8):
        sep = ckks.add(P, sep, ckks.rotate(P, keys, ct, r))
    q = P.q[: ct.level + 1]
    for c in range(2):
        a = ckks.crt_centered(one.c[c], q)
        b = ckks.crt_centered(sep.c[c], q)
        d = max(abs(int(x) - int(y)) for x, y in zip(a, b))
        assert 0 < d <= 3 * (P.alpha + 1)
    assert np.max(np.abs(ckks.decrypt(P, keys, one) - ckks.decrypt(P, keys, sep))) < 2.0 ** -25


def test_oracle_rank_over_pairs_decrypts_to_ranks():
    """With the pair-sum rotation keys every chain of the rank runs two steps at a time
    (has_rot), and the encrypted rank decrypts to the brute-force ranks."""
    P = helpers.oracle_params("ord")
    N = 8
    keys = ckks.keygen(P, 74, helpers.galois_elts(P, helpers.rotation_set(N)))
    Bo = C.OracleCkks(P, keys)
    assert all(len(st) == 3 for st in C.chain_pairs(Bo, C.repl_r_amounts(N))[:1])
    v = inputs.gap_vector(N, 0.05, 75)
    R = C.rank(Bo, ckks.encrypt(P, keys, v, 75), N, 2, 1)
    assert np.max(np.abs(ckks.decrypt(P, keys, R)[:N] - C.brute_fractional_rank(v))) < 0.25
