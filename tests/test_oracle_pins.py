"""Pins of the oracle's comparator stages and of the product's single rounding
against facts outside the oracle.

* The composite comparator (Sec. 2.2): each odd degree-7 stage, as the oracle's
  depth-3 schedule evaluates it, equals the paper's printed f(x) = (35x - 35x^3 +
  21x^5 - 5x^7) / 2^4 and g(x) = (4589x - 16577x^3 + 25614x^5 - 12860x^7) / 2^10,
  built here from those integer numerators; f is also the closed form
  f' = (35/16)(1 - x^2)^3 integrated from 0; the last stage's folding of 1/2 gives
  (f^df(g^dg(x)) + 1)/2.
* The single rounding of a product (multiple of q_l P decided in IEEE double): over a
  whole ring of the 128-element parameter set, the decision equals exact big-integer
  rounding of u / (q_l P) everywhere except within the double sum's error bound of a
  half-integer, and planted half-integer cases land on one of the two neighbours.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ckks, circuits as C
from tests import helpers

# The paper's printed numerators and denominators (Sec. 2.2).
F_NUM, F_DEN = (35, -35, 21, -5), 2 ** 4
G_NUM, G_DEN = (4589, -16577, 25614, -12860), 2 ** 10


def _printed(num, den, x):
    """sum_k num_k x^(2k+1) / den in float64 (Horner in x^2)."""
    x2 = x * x
    acc = np.zeros_like(x)
    for a in reversed(num):
        acc = acc * x2 + a
    return acc * x / den


def _plain_stage(coeffs, x):
    Bp = C.PlainSlots(x.size, 3)
    return Bp.values(C.poly7(Bp, Bp.fresh(x), coeffs))


GRID = np.linspace(-1.0, 1.0, 8193)


@pytest.mark.parametrize("name", ["f", "g"])
def test_stage_schedule_is_the_printed_polynomial(name):
    """The depth-3 schedule p = (c5 x + c7 x^3) x^4 + (c3/c7)(c7 x^3) + c1 x with the
    oracle's stage coefficients reproduces the printed polynomial on a dense grid."""
    coeffs = C.F_COEFFS if name == "f" else C.G_COEFFS
    num, den = (F_NUM, F_DEN) if name == "f" else (G_NUM, G_DEN)
    got = _plain_stage(coeffs, GRID)
    assert np.max(np.abs(got - _printed(num, den, GRID))) < 1e-12
    # the coefficients themselves, exactly
    assert [Fraction(c).limit_denominator(den) * den for c in coeffs] == list(num)
    assert all(c * den == a for c, a in zip(coeffs, num))


def test_f_is_the_integral_of_its_closed_form_derivative():
    """f' = (35/16)(1 - x^2)^3: f(x) = (35/16)(x - x^3 + 3x^5/5 - x^7/7), a fact
    independent of the printed numerators; f(+-1) = +-1 and f odd."""
    closed = (35.0 / 16) * (GRID - GRID ** 3 + 0.6 * GRID ** 5 - GRID ** 7 / 7.0)
    got = _plain_stage(C.F_COEFFS, GRID)
    assert np.max(np.abs(got - closed)) < 1e-12
    assert abs(got[-1] - 1.0) < 1e-15 and abs(got[0] + 1.0) < 1e-15
    assert np.max(np.abs(got + got[::-1])) < 1e-15


def test_g_maps_the_interval_into_itself_and_steepens():
    """g is odd with g(1) = 766/1024 and |g(x)| <= 1 on [-1, 1], and g'(0) = 4589/1024 > f'(0):
    the steeper first stages the composite applies before f (Sec. 2.2)."""
    got = _plain_stage(C.G_COEFFS, GRID)
    assert abs(got[-1] - 766 / 1024) < 1e-15
    assert np.max(np.abs(got)) <= 1.0 + 1e-12
    h = 1e-6
    slope = _plain_stage(C.G_COEFFS, np.array([h]))[0] / h
    assert abs(slope - 4589 / 1024) < 1e-6


@pytest.mark.parametrize("dg, df", [(2, 1), (3, 2), (4, 2), (1, 1)])
def test_cmp_stages_fold_the_half(dg, df):
    """Cmp over the oracle's stages = (f^df(g^dg(x)) + 1) / 2 with f, g from the printed
    integers; Cmp(0) = 1/2 exactly (odd stages)."""
    Bp = C.PlainSlots(GRID.size, 3 * (dg + df))
    got = Bp.values(C.cmp(Bp, Bp.fresh(GRID), dg, df))
    y = GRID.copy()
    for _ in range(dg):
        y = _printed(G_NUM, G_DEN, y)
    for _ in range(df):
        y = _printed(F_NUM, F_DEN, y)
    assert np.max(np.abs(got - (y + 1.0) / 2.0)) < 1e-11
    assert got[GRID.size // 2] == 0.5
    assert len(C.cmp_stages(dg, df)) == dg + df


# --------------------------------------------------------------------------
# The product's single rounding over a whole ring
# --------------------------------------------------------------------------
# The double sum f^ = sum_k fl(fl(y_k) * fl(1/s_k)) over A + 1 terms, each below 1,
# differs from t = sum_k y_k / s_k by at most (A+1)(A+4) 2^-53 (three roundings a
# term, A additions of partial sums below A + 1, one addition of 1/2): for A = 3
# special primes that is 28 * 2^-53 < 2^-48.  So floor(f^ + 1/2) = round(t) unless
# the fractional part of t lies within 2^-48 of 1/2.
HALF_MARGIN = 2.0 ** -48


def _exact_multiple(u, src):
    """For residues u [k][n] over the primes src: X = sum_k y_k S/s_k (y_k = u_k (S/s_k)^-1
    mod s_k), the integer nearest to X / S rounded half up, and the distance of X / S
    from the nearest half-integer, in units of 1 (Python integers)."""
    S = math.prod(int(s) for s in src)
    X = np.zeros(u.shape[1], dtype=object)
    for k, s in enumerate(src):
        s = int(s)
        Sk = S // s
        inv = pow(Sk % s, -1, s)
        y = (u[k].astype(object) * inv) % s
        X = X + y * Sk
    v = (2 * X + S) // (2 * S)
    frac = [Fraction(int(x) % S, S) for x in X]
    dist = np.array([abs(float(f - Fraction(1, 2))) for f in frac])
    return X, v, S, dist


def test_rounded_conversion_matches_exact_rounding_on_a_full_ring():
    """128-element parameter set (n = 2^16), top level: sources {q_27, p_0, p_1, p_2},
    destinations q_0 .. q_26.  On a whole ring of uniform residues the double decision
    equals exact rounding of X / S at every coefficient (none lies within 2^-48 of a
    half-integer); on planted coefficients with X / S within 2^-200 of a half-integer,
    the result is one of the two neighbouring multiples."""
    P = helpers.oracle_params("cfg2")
    lvl = P.L
    src = [int(P.q[lvl])] + [int(p) for p in P.p]
    dst = [int(q) for q in P.q[:lvl]]
    rng = np.random.default_rng(2412)
    n = P.n
    u = np.stack([rng.integers(0, s, n, dtype=np.uint64) for s in src])
    # plant near-half coefficients: X = (S - 1)/2 + d for small d (S is odd)
    S = math.prod(src)
    planted = list(range(0, n, 4099))
    for t, k in enumerate(planted):
        Xk = (S - 1) // 2 + (t % 3)   # fractional part 1/2 - 1/(2S), 1/2 + 1/(2S), ...
        for i, s in enumerate(src):   # the residues of X_k: X = X_k + j S, j in [0, A]
            u[i, k] = Xk % s
    w = ckks.base_conv_rounded(u, src, dst)
    X, v, S, dist = _exact_multiple(u, src)
    mismatched = []
    for m, t in enumerate(dst):
        exact = np.array([int((int(x) - int(vv) * S) % t) for x, vv in zip(X, v)], dtype=np.uint64)
        bad = np.nonzero(exact != w[m])[0]
        mismatched.extend(bad.tolist())
        # every disagreement is the other neighbour: X - (v -+ 1) S
        for k in bad:
            alt = {int((int(X[k]) - (int(v[k]) + d) * S) % t) for d in (-1, 1)}
            assert int(w[m, k]) in alt
    mismatched = sorted(set(mismatched))
    assert all(dist[k] < HALF_MARGIN for k in mismatched), [(k, dist[k]) for k in mismatched]
    assert set(mismatched) <= set(planted)
    planted_set = set(planted)
    far = [k for k in range(n) if k not in planted_set]
    assert float(np.min(dist[far])) >= HALF_MARGIN
