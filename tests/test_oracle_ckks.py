"""Pins for the oracle's homomorphic operations on a small ring (n = 2^10):
decryptions against the closed-form slot results, and the integer identities of
rescaling, ModDown and key switching checked with Python big integers."""
import math

import numpy as np
import pytest

from oracle import ckks

LOG_N = 10
N_RING = 1 << LOG_N


@pytest.fixture(scope="module")
def setup():
    P = ckks.gen_params(LOG_N, 6, 60, 40, 2, 61, 2)
    rots = [1, 3, 5, P.slots - 3, 17]
    keys = ckks.keygen(P, 42, [ckks.galois_left(r, P.n) for r in rots])
    rng = np.random.default_rng(9)
    z1 = rng.uniform(-1, 1, P.slots)
    z2 = rng.uniform(-1, 1, P.slots)
    c1 = ckks.encrypt(P, keys, z1, 1)
    c2 = ckks.encrypt(P, keys, z2, 2)
    return P, keys, z1, z2, c1, c2, rots


def test_encrypt_decrypt(setup):
    P, keys, z1, _, c1, _, _ = setup
    assert np.max(np.abs(ckks.decrypt(P, keys, c1) - z1)) < 2.0 ** -25


def test_rotation_is_cyclic_shift(setup):
    P, keys, z1, _, c1, _, rots = setup
    for r in rots:
        got = ckks.decrypt(P, keys, ckks.rotate(P, keys, c1, r))
        assert np.max(np.abs(got - np.roll(z1, -r))) < 2.0 ** -20, r


def test_add_sub_neg_const(setup):
    P, keys, z1, z2, c1, c2, _ = setup
    assert np.max(np.abs(ckks.decrypt(P, keys, ckks.add(P, c1, c2)) - (z1 + z2))) < 2.0 ** -24
    assert np.max(np.abs(ckks.decrypt(P, keys, ckks.sub(P, c1, c2)) - (z1 - z2))) < 2.0 ** -24
    assert np.max(np.abs(ckks.decrypt(P, keys, ckks.neg(P, c1)) + z1)) < 2.0 ** -24
    assert np.max(np.abs(ckks.decrypt(P, keys, ckks.add_const(P, c1, 0.75)) - (z1 + 0.75))) < 2.0 ** -24


def test_mul_and_levels(setup):
    P, keys, z1, z2, c1, c2, _ = setup
    m = ckks.mul(P, keys, c1, c2)
    assert m.level == P.L - 1
    assert np.max(np.abs(ckks.decrypt(P, keys, m) - z1 * z2)) < 2.0 ** -20
    m2 = ckks.mul(P, keys, m, m)
    assert np.max(np.abs(ckks.decrypt(P, keys, m2) - (z1 * z2) ** 2)) < 2.0 ** -18


def test_mul_scalar_plain_level_down(setup):
    P, keys, z1, _, c1, _, _ = setup
    got = ckks.decrypt(P, keys, ckks.mul_scalar(P, c1, -3.25))
    assert np.max(np.abs(got - (-3.25 * z1))) < 2.0 ** -20
    mask = (np.arange(P.slots) % 3 == 0).astype(float)
    got = ckks.decrypt(P, keys, ckks.mul_plain(P, c1, ckks.encode_unscaled(mask, P.n)))
    assert np.max(np.abs(got - z1 * mask)) < 2.0 ** -20
    d = ckks.level_down(P, c1, P.L - 3)
    assert d.level == P.L - 3
    assert np.max(np.abs(ckks.decrypt(P, keys, d) - z1)) < 2.0 ** -20


def _crt(res, primes):
    return ckks.crt_centered(np.asarray(res, dtype=np.uint64), primes)


def test_rescale_is_rounded_division(setup):
    P, keys, _, _, c1, _, _ = setup
    out = ckks.rescale(P, c1)
    lvl = c1.level
    ql = P.q[lvl]
    Qin = math.prod(P.q[: lvl + 1])
    for c in range(2):
        x = _crt(c1.c[c], P.q[: lvl + 1])
        y = _crt(out.c[c], P.q[:lvl])
        for k in range(0, P.n, 41):
            diff = (int(y[k]) * ql - int(x[k])) % Qin
            if diff > Qin // 2:
                diff -= Qin
            # y * q_l = x - r with r = x mod q_l centred into (-q_l/2, q_l/2]
            r = int(x[k]) % ql
            if r > (ql - 1) // 2:
                r -= ql
            assert diff == -r


def test_mod_down_divides_by_P(setup):
    P, _, _, _, _, _, _ = setup
    lvl = 3
    primes = P.qp(lvl)
    rng = np.random.default_rng(4)
    u = np.stack([rng.integers(0, q, P.n, dtype=np.uint64) for q in primes])
    out = ckks.mod_down(P, u, lvl)
    Pp = math.prod(P.p)
    Q = math.prod(P.q[: lvl + 1])
    U = ckks.crt_centered(u, primes)
    Y = ckks.crt_centered(out, P.q[: lvl + 1])
    for k in range(0, P.n, 29):
        # out = (u - ([u]_P + e P)) / P with 0 <= e < alpha: |out - u/P| <= alpha + 1 (mod Q)
        d = (int(Y[k]) * Pp - int(U[k])) % (Q * Pp)
        if d > (Q * Pp) // 2:
            d -= Q * Pp
        assert abs(d) <= (P.alpha + 1) * Pp


def test_mod_down_is_unbiased(setup):
    """out*P - u has mean ~0 over coefficients: the centred conversion removes the
    positive bias (alpha-1)/2 * P of an uncentred fast conversion."""
    P, _, _, _, _, _, _ = setup
    lvl = 3
    primes = P.qp(lvl)
    rng = np.random.default_rng(8)
    u = np.stack([rng.integers(0, q, P.n, dtype=np.uint64) for q in primes])
    out = ckks.mod_down(P, u, lvl)
    Pp = math.prod(P.p)
    Q = math.prod(P.q[: lvl + 1])
    U = ckks.crt_centered(u, primes)
    Y = ckks.crt_centered(out, P.q[: lvl + 1])
    d = []
    for k in range(P.n):
        x = (int(Y[k]) * Pp - int(U[k])) % (Q * Pp)
        if x > (Q * Pp) // 2:
            x -= Q * Pp
        d.append(x / Pp)
    assert abs(np.mean(d)) < 0.1
    assert max(abs(x) for x in d) <= P.alpha


def test_rotation_error_is_unbiased(setup):
    """After eight rotations the decrypted coefficients minus the encoded expected
    slots have mean ~0.  (A constant coefficient bias b decodes to an error of about
    b 2n/pi at slot 0; an uncentred ModDown gives b ~ (alpha-1)/2 * sum(s) per switch.)"""
    P, keys, z1, _, c1, _, rots = setup
    x = c1
    tot = 0
    for r in (1, 5, 17, 3) * 2:
        x = ckks.rotate(P, keys, x, r)
        tot += r
    got = ckks.decrypt_coeffs(P, keys, x).astype(np.float64)
    expect = ckks.encode(np.roll(z1, -tot), P.scales[x.level], P.n).astype(np.float64)
    assert abs(np.mean(got - expect)) < 5.0


def test_key_switch_relation(setup):
    """KS(d) = (k0, k1) with k0 + k1 s = d s^2 + small error (relinearisation key)."""
    P, keys, _, _, _, _, _ = setup
    for lvl in (P.L, 2):
        q = P.q[: lvl + 1]
        rng = np.random.default_rng(lvl)
        d = np.stack([rng.integers(0, qi, P.n, dtype=np.uint64) for qi in q])
        k0, k1 = ckks.key_switch(P, d, keys.rlk, lvl)
        s = ckks.to_residues(keys.s, q)
        lhs = ckks.add_mod(k0, ckks.ring_mul(k1, s, q), q)
        rhs = ckks.ring_mul(d, ckks.ring_mul(s, s, q), q)
        err = ckks.crt_centered(ckks.sub_mod(lhs, rhs, q), q)
        assert max(abs(int(e)) for e in err) < 2 ** 24


def test_mod_down_rescale_divides_by_P_ql(setup):
    """Fused ModDown + rescale: out = round(u / (P q_l)), i.e. out (P q_l) - u is the
    centred representative of u mod P q_l, |.| <= P q_l / 2 (checked with Python
    integers on sampled coefficients)."""
    P, _, _, _, _, _, _ = setup
    for lvl in (3, P.L):
        primes = P.qp(lvl)
        rng = np.random.default_rng(40 + lvl)
        u = np.stack([rng.integers(0, q, P.n, dtype=np.uint64) for q in primes])
        out = ckks.mod_down_rescale(P, u, lvl)
        assert out.shape == (lvl, P.n)
        S = math.prod(P.p) * int(P.q[lvl])
        Q = math.prod(P.q[:lvl])
        U = ckks.crt_centered(u, primes)
        Y = ckks.crt_centered(out, P.q[:lvl])
        for k in range(0, P.n, 23):
            d = (int(Y[k]) * S - int(U[k])) % (Q * S)
            if d > (Q * S) // 2:
                d -= Q * S
            assert abs(d) <= S // 2
            assert d == (-int(U[k])) % S or d == (-int(U[k])) % S - S


def test_fused_product_matches_two_step(setup):
    """The product's single rounding and ModDown-then-rescale differ by at most a
    few units in the last place: decryptions agree far below the noise."""
    P, keys, z1, z2, c1, c2, _ = setup
    lvl = c1.level
    q = P.q[: lvl + 1]
    d0 = ckks.ring_mul(c1.c[0], c2.c[0], q)
    d1 = ckks.ring_mac(np.stack([c1.c[0], c1.c[1]]), np.stack([c2.c[1], c2.c[0]]), q)
    d2 = ckks.ring_mul(c1.c[1], c2.c[1], q)
    k0, k1 = ckks.key_switch(P, d2, keys.rlk, lvl)
    two = ckks.rescale(P, ckks.Ct(np.stack([ckks.add_mod(d0, k0, q), ckks.add_mod(d1, k1, q)]), lvl))
    fused = ckks.mul(P, keys, c1, c2)
    for c in range(2):
        a = ckks.crt_centered(two.c[c], P.q[:lvl])
        b = ckks.crt_centered(fused.c[c], P.q[:lvl])
        assert max(abs(int(x) - int(y)) for x, y in zip(a[::37], b[::37])) <= 2
    assert np.max(np.abs(ckks.decrypt(P, keys, fused) - z1 * z2)) < 2.0 ** -20
