"""Pins for the oracle's modular arithmetic, prime chain, ring product, basis
conversion and automorphism - each checked against something other than the
oracle itself (sympy primality, Python big integers, direct polynomial
evaluation)."""
import math

import numpy as np
import pytest

from oracle import ckks

sympy = pytest.importorskip("sympy")

CONFIGS = {
    "n2^13_14x40": (13, 14, 40, 40, 1, 61, 1),
    "n2^16_28limbs": (16, 28, 60, 45, 3, 61, 3),
    "n2^16_34limbs": (16, 34, 60, 45, 3, 61, 3),
    # every prime k 2^32 + 1 (prime_form 1)
    "n2^16_28limbs_k32": (16, 28, 60, 45, 3, 61, 3, 1),
    "n2^16_34limbs_k32": (16, 34, 60, 45, 3, 61, 3, 1),
    "n2^15_34limbs_k32": (15, 34, 60, 45, 3, 61, 3, 1),
}


def test_is_prime_matches_sympy():
    rng = np.random.default_rng(0)
    xs = list(range(0, 3000))
    xs += [int(v) for v in rng.integers(2 ** 40, 2 ** 61, 400, dtype=np.uint64)]
    # strong pseudoprimes to several small bases
    xs += [3215031751, 2152302898747, 3474749660383, 341550071728321, 3825123056546413051]
    for x in xs:
        assert ckks.is_prime(x) == sympy.isprime(x), x


@pytest.mark.parametrize("name", list(CONFIGS))
def test_prime_chain(name):
    log_n, n_q, b0, logd, alpha, bp, dsize = CONFIGS[name][:7]
    form = CONFIGS[name][7] if len(CONFIGS[name]) > 7 else 0
    P = ckks.gen_params(*CONFIGS[name])
    m = (1 << 32) if form else 2 << log_n
    assert m % (2 << log_n) == 0
    allp = list(P.q) + list(P.p)
    assert len(set(allp)) == len(allp)
    for x in allp:
        assert sympy.isprime(x) and x % m == 1
    # q_0: no admissible prime between q_0 and 2^b0
    c = P.q[0] + m
    while c < (1 << b0):
        assert not sympy.isprime(c)
        c += m
    # specials: the largest admissible primes below 2^bp not already in the chain
    c = ((1 << bp) - 2) // m * m + 1
    expect = []
    while len(expect) < alpha:
        if sympy.isprime(c) and c not in P.q:
            expect.append(c)
        c -= m
    assert list(P.p) == expect
    # scale chain: Delta_L = 2^logd, Delta_{l-1} = Delta_l^2 / q_l, q_l nearest floor(Delta_l^2 / 2^logd)
    assert P.scales[P.L] == 2.0 ** logd
    used = {P.q[0]}
    for lvl in range(P.L, 0, -1):
        assert P.scales[lvl - 1] == P.scales[lvl] * P.scales[lvl] / float(P.q[lvl])
        target = math.floor(P.scales[lvl] * P.scales[lvl] / 2.0 ** logd)
        d = abs(P.q[lvl] - target)
        # no unused admissible prime strictly closer (or equally close and smaller)
        lo = (target - d) // m * m + 1
        c = lo
        while c <= target + d:
            if c % m == 1 and c != P.q[lvl] and c not in used and sympy.isprime(c):
                dc = abs(c - target)
                assert dc > d or (dc == d and c > P.q[lvl]), (lvl, c, P.q[lvl])
            c += m
        used.add(P.q[lvl])
    # canonical scales near 2^logd: the candidates = 1 mod 2n are dense near 2^45; those
    # = 1 mod 2^32 are 2^32 apart and prime about one in 16, so the nearest lie within
    # a few percent
    for s in P.scales:
        assert abs(s / 2.0 ** logd - 1.0) < (0.05 if form else 2.0 ** -15)


def test_security_budgets():
    # log QP of the n = 2^16 sets against the 128-bit ternary-secret bound of the HE
    # standard for n = 2^16 (1772 bits); config 2 additionally within 1550.
    assert ckks.gen_params(*CONFIGS["n2^16_28limbs"]).log_qp() <= 1550
    assert ckks.gen_params(*CONFIGS["n2^16_34limbs"]).log_qp() <= 1772
    assert ckks.gen_params(*CONFIGS["n2^16_28limbs_k32"]).log_qp() <= 1550
    assert ckks.gen_params(*CONFIGS["n2^16_34limbs_k32"]).log_qp() <= 1772


def _negacyclic_bigint(a, b, q):
    n = len(a)
    full = np.convolve(np.array(a, dtype=object), np.array(b, dtype=object))
    out = [0] * n
    for k, v in enumerate(full):
        if k < n:
            out[k] += v
        else:
            out[k - n] -= v
    return [x % q for x in out]


@pytest.mark.parametrize("log_n", [4, 6, 8, 10])
def test_ring_product_matches_schoolbook(log_n):
    n = 1 << log_n
    P = ckks.gen_params(log_n, 3, 50, 40, 1, 61, 1)
    rng = np.random.default_rng(log_n)
    primes = list(P.q) + list(P.p)
    a = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in primes])
    b = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in primes])
    # boundary residues
    a[:, 0] = np.array(primes, dtype=np.uint64) - 1
    b[:, -1] = np.array(primes, dtype=np.uint64) - 1
    got = ckks.ring_mul(a, b, primes)
    for i, q in enumerate(primes):
        ref = _negacyclic_bigint([int(x) for x in a[i]], [int(x) for x in b[i]], q)
        assert [int(x) for x in got[i]] == ref


def test_ring_mac_is_sum_of_products():
    n = 64
    P = ckks.gen_params(6, 2, 50, 40, 1, 61, 1)
    rng = np.random.default_rng(3)
    primes = list(P.q)
    A = np.stack([np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in primes]) for _ in range(3)])
    Bm = np.stack([np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in primes]) for _ in range(3)])
    got = ckks.ring_mac(A, Bm, primes)
    for i, q in enumerate(primes):
        ref = [0] * n
        for t in range(3):
            r = _negacyclic_bigint([int(x) for x in A[t, i]], [int(x) for x in Bm[t, i]], q)
            ref = [(u + v) % q for u, v in zip(ref, r)]
        assert [int(x) for x in got[i]] == ref


@pytest.mark.parametrize("n_src", [1, 2, 3])
def test_fast_base_conv_is_crt_plus_small_multiple(n_src):
    P = ckks.gen_params(10, 6, 60, 45, 3, 61, 3)
    src = P.q[1:1 + n_src]
    dst = list(P.q) + list(P.p)
    n = 1 << 10
    rng = np.random.default_rng(n_src)
    x = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in src])
    x[:, 0] = 0
    x[:, 1] = np.array(src, dtype=np.uint64) - 1
    out = ckks.fast_base_conv(x, src, dst)
    D = math.prod(src)
    for k in range(0, n, 37):
        X = sympy.ntheory.modular.crt(src, [int(v) for v in x[:, k]])[0] % D
        us = set()
        for m_, t in enumerate(dst):
            if D % t == 0:
                assert int(out[m_, k]) == X % t
                continue
            u = ((int(out[m_, k]) - X) * pow(D % t, -1, t)) % t
            us.add(u)
        assert len(us) == 1 and 0 <= us.pop() < n_src


def _eval_poly(coeffs, x, q):
    acc = 0
    for c in reversed([int(v) for v in coeffs]):
        acc = (acc * x + c) % q
    return acc


def test_automorphism_is_evaluation_permutation():
    log_n = 5
    n = 1 << log_n
    P = ckks.gen_params(log_n, 2, 40, 30, 1, 50, 1)
    q = P.q[0]
    # a primitive 2n-th root of unity found independently of the oracle
    g0 = sympy.primitive_root(q)
    psi = pow(g0, (q - 1) // (2 * n), q)
    assert pow(psi, n, q) == q - 1
    rng = np.random.default_rng(5)
    a = rng.integers(0, q, n, dtype=np.uint64)[None]
    for r in (1, 3, 7, n // 2 - 1):
        g = ckks.galois_left(r, n)
        b = ckks.automorphism(a, g, [q])
        for e in range(1, 2 * n, 2):
            assert _eval_poly(b[0], pow(psi, e, q), q) == _eval_poly(a[0], pow(psi, e * g, q), q)


def test_rha_rounding():
    xs = np.array([0.5, -0.5, 1.5, 2.5, -2.5, 0.49999999999999994, -0.49999999999999994,
                   1.4999999999999998, 3.0, -7.25, 2.0 ** 52 + 1, -(2.0 ** 52) - 1])
    expect = [1, -1, 2, 3, -3, 0, 0, 1, 3, -7, 2 ** 52 + 1, -(2 ** 52) - 1]
    assert list(ckks.rha(xs)) == expect
    assert [ckks.rha_scalar(float(x)) for x in xs] == expect


# SplitMix64 reference outputs for seed 1234567 (the generator's published test
# vector: the first five values of the stream).
SPLITMIX64_1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                      4593380528125082431, 16408922859458223821]


def test_seeded_generator_is_splitmix64():
    """The key generator's stream is SplitMix64: word i of a one-prime, one-digit key
    of length 5 is the high word of x_i q for the published outputs x_i."""
    from oracle import _lib
    q = (1 << 61) - 1
    out = np.empty(5, dtype=np.uint64)
    _lib.lib().orc_seeded_key_a(1234567, 0, 1, _lib.ptr(np.array([q], dtype=np.uint64)), 1, 5, _lib.ptr(out))
    assert [int(v) for v in out] == [(x * q) >> 64 for x in SPLITMIX64_1234567]


def test_seeded_key_a_evaluates_to_the_stream():
    """seeded_key_a's coefficients evaluate, at psi^(2 brev(i) + 1), to the stream value
    times 2^-64 (Horner with Python integers, sampled i; psi the first c^((q-1)/2n)
    of order 2n): pins the order, the root and the Montgomery reading."""
    from oracle import _lib
    P = ckks.gen_params(8, 3, 50, 40, 1, 55, 1)
    primes = P.qp(P.L)
    seed, j = 987654321, 1
    a = ckks.seeded_key_a(P, seed, j)
    T = len(primes)
    raw = np.empty((T, P.n), dtype=np.uint64)
    _lib.lib().orc_seeded_key_a(seed, j, T, _lib.ptr(np.array(primes, dtype=np.uint64)), T, P.n, _lib.ptr(raw))
    logn = P.n.bit_length() - 1
    for p, q in enumerate(primes):
        q = int(q)
        c = 2
        while True:
            psi = pow(c, (q - 1) // (2 * P.n), q)
            if pow(psi, P.n, q) == q - 1:
                break
            c += 1
        rinv = pow(pow(2, 64, q), -1, q)
        for i in (0, 1, 5, 77, P.n - 1):
            x = pow(psi, 2 * int(format(i, f"0{logn}b")[::-1], 2) + 1, q)
            acc = 0
            for coef in reversed(a[p].tolist()):
                acc = (acc * x + int(coef)) % q
            assert acc == int(raw[p, i]) * rinv % q
