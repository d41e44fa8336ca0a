"""Plain RNS-CKKS oracle (Sec. 2.1 of the paper: ring Z_q[x]/(x^n+1), n/2 slots,
addition, multiplication and slot rotation).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  It shares no code with the CUDA library.

Every polynomial is kept in the coefficient domain as residues in [0, q).  A
ciphertext at level l is an array ``c[2][l+1][n]`` (uint64) over the primes
q_0..q_l; its scale is the canonical scale Delta_l of that level.  The paper
fixes only the scheme; the conventions below are the readings this project
fixes (each is stated once here and implemented independently by the CUDA
library):

  moduli     q_0 = largest prime < 2^b0 with q = 1 mod 2n; q_L..q_1 chosen top
             down, q_l the unused prime = 1 mod 2n nearest floor(Delta_l^2 / 2^logD)
             (ties to the smaller), Delta_L = 2^logD, Delta_{l-1} = Delta_l^2 / q_l;
             specials p_0 > p_1 > ... the largest unused primes < 2^bp, = 1 mod 2n.
             prime_form 1: the same rules with every "= 1 mod 2n" read "= 1 mod 2^32"
             (primes k 2^32 + 1; 2n divides 2^32, so they stay NTT-friendly).
  encoding   slot j <-> evaluation at zeta^(5^j), zeta = exp(i pi / n); a plaintext
             at scale s has coefficients rha(s * u_k) where u is the real
             polynomial with those evaluations and rha rounds half away from 0.
  digits     digit j at level l covers limbs [j*dsize, min((j+1)*dsize, l+1)).
  ModUp      fast basis conversion of one digit without correction.
  KS         ModUp every digit, (for a rotation) apply the automorphism to the
             lifted digits, multiply-accumulate with the key over Q_l u P, ModDown.
  ModDown    fast basis conversion of the P part to Q_l with centred terms
             (y_k in (-p_k/2, p_k/2]), subtract, times P^-1.
  rescale    centred lift of the last residue into (-q_l/2, q_l/2], subtract,
             times q_l^-1.
  mul        (x0 y0, x0 y1 + x1 y0, x1 y1), relinearise x1 y1, rescale.
  scalar c   multiply by rha(c * s), s = Delta_{l-1} q_l / Delta_l, rescale.
  plaintext  multiply by the plaintext encoded at that same s, rescale.
  add const  add rha(c * Delta_l) to coefficient 0 of c0.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import _lib
from ._lib import ptr, u64


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------
def is_prime(x: int) -> bool:
    return bool(_lib.lib().orc_is_prime(int(x)))


def _largest_prime_below(bound: int, m: int, used: set) -> int:
    k = (bound - 2) // m
    while True:
        c = k * m + 1
        if c not in used and is_prime(c):
            return c
        k -= 1


def _nearest_prime(c: int, m: int, used: set) -> int:
    """Prime = 1 mod m nearest to the integer c, ties to the smaller, not in used."""
    lo = ((c - 1) // m) * m + 1  # largest candidate <= c
    hi = lo + m                   # smallest candidate > c
    while True:
        if c - lo <= hi - c:
            if lo > 2 and lo not in used and is_prime(lo):
                return lo
            lo -= m
        else:
            if hi not in used and is_prime(hi):
                return hi
            hi += m


@dataclass
class Params:
    log_n: int
    q: list            # q_0 .. q_L
    p: list            # special primes
    scales: list       # Delta_0 .. Delta_L (doubles)
    dsize: int
    log_scale: int

    @property
    def n(self) -> int:
        return 1 << self.log_n

    @property
    def slots(self) -> int:
        return self.n // 2

    @property
    def L(self) -> int:
        return len(self.q) - 1

    @property
    def alpha(self) -> int:
        return len(self.p)

    def beta(self, level: int) -> int:
        return -(-(level + 1) // self.dsize)

    def qp(self, level: int) -> list:
        return list(self.q[: level + 1]) + list(self.p)

    def log_qp(self) -> float:
        return sum(math.log2(x) for x in self.q) + sum(math.log2(x) for x in self.p)


def gen_params(log_n: int, n_q: int, log_q0: int, log_scale: int, n_special: int,
               log_special: int, dsize: int, prime_form: int = 0) -> Params:
    n = 1 << log_n
    m = (1 << 32) if prime_form else 2 * n
    used: set = set()
    q0 = _largest_prime_below(1 << log_q0, m, used)
    used.add(q0)
    L = n_q - 1
    q = [0] * (L + 1)
    q[0] = q0
    scales = [0.0] * (L + 1)
    scales[L] = float(2 ** log_scale)
    for lvl in range(L, 0, -1):
        target = scales[lvl] * scales[lvl] / float(2 ** log_scale)
        ql = _nearest_prime(int(math.floor(target)), m, used)
        used.add(ql)
        q[lvl] = ql
        scales[lvl - 1] = (scales[lvl] * scales[lvl]) / float(ql)
    p = []
    bound = 1 << log_special
    for _ in range(n_special):
        pk = _largest_prime_below(bound, m, used)
        used.add(pk)
        p.append(pk)
        bound = pk
    return Params(log_n=log_n, q=q, p=p, scales=scales, dsize=dsize, log_scale=log_scale)


# --------------------------------------------------------------------------
# Rounding and residues
# --------------------------------------------------------------------------
def rha(x):
    """Round half away from zero, exactly (x - trunc(x) is exact in binary64)."""
    x = np.asarray(x, dtype=np.float64)
    t = np.trunc(x)
    frac = x - t
    return (t + np.where(np.abs(frac) >= 0.5, np.sign(x), 0.0)).astype(np.int64)


def rha_scalar(x: float) -> int:
    t = math.trunc(x)
    frac = x - t
    if abs(frac) >= 0.5:
        t += 1 if x > 0 else -1
    return int(t)


def to_residues(m: np.ndarray, primes) -> np.ndarray:
    """Signed int64 coefficients -> residues [len(primes)][n] in [0, q)."""
    m = np.asarray(m, dtype=np.int64)
    out = np.empty((len(primes), m.shape[-1]), dtype=np.uint64)
    for i, qi in enumerate(primes):
        out[i] = np.mod(m, np.int64(qi)).astype(np.uint64)
    return out


def _qcol(primes) -> np.ndarray:
    return np.asarray(primes, dtype=np.uint64).reshape(-1, 1)


def add_mod(a, b, primes):
    return (a + b) % _qcol(primes)


def sub_mod(a, b, primes):
    return (a + (_qcol(primes) - b)) % _qcol(primes)


def neg_mod(a, primes):
    return (_qcol(primes) - a) % _qcol(primes)


def mul_scalar_mod(a, consts, primes):
    a = u64(a)
    out = np.empty_like(a)
    _lib.lib().orc_mul_scalar(ptr(a), ptr(u64(consts)), ptr(out), a.shape[0], a.shape[1], ptr(u64(primes)))
    return out


def ring_mac(a_terms, b_terms, primes):
    """sum_t a_t * b_t in prod_l Z_{q_l}[x]/(x^n+1); a_terms, b_terms: [T][limbs][n]."""
    a = u64(a_terms)
    b = u64(b_terms)
    T, limbs, n = a.shape
    assert b.shape == (T, limbs, n), (a.shape, b.shape)
    out = np.empty((limbs, n), dtype=np.uint64)
    _lib.lib().orc_ring_mac(ptr(a), limbs * n, ptr(b), limbs * n, T, ptr(out), limbs, n, ptr(u64(primes)))
    return out


def ring_mul(a, b, primes):
    return ring_mac(u64(a)[None], u64(b)[None], primes)


def fast_base_conv(x, src, dst):
    x = u64(x)
    out = np.empty((len(dst), x.shape[1]), dtype=np.uint64)
    _lib.lib().orc_fast_base_conv(ptr(x), x.shape[1], ptr(u64(src)), len(src), ptr(u64(dst)), len(dst), ptr(out))
    return out


def fast_base_conv_centered(x, src, dst):
    """Fast basis conversion with each term y_i taken in (-s_i/2, s_i/2]."""
    x = u64(x)
    out = np.empty((len(dst), x.shape[1]), dtype=np.uint64)
    _lib.lib().orc_fast_base_conv_centered(ptr(x), x.shape[1], ptr(u64(src)), len(src), ptr(u64(dst)), len(dst),
                                           ptr(out))
    return out


def automorphism(a, g: int, primes):
    """X -> X^g on each residue polynomial: coefficient k moves to k*g mod 2n,
    negated when that index is >= n (because X^n = -1)."""
    a = u64(a)
    n = a.shape[-1]
    k = np.arange(n, dtype=np.int64)
    dest = (k * (g % (2 * n))) % (2 * n)
    neg = dest >= n
    dest = dest % n
    out = np.empty_like(a)
    q = _qcol(primes)
    out[:, dest] = np.where(neg[None, :], (q - a) % q, a)
    return out


def crt_centered(res, primes):
    """Residues [limbs][n] -> centred integers (Python ints, object array)."""
    Q = 1
    for qi in primes:
        Q *= int(qi)
    acc = np.zeros(res.shape[1], dtype=object)
    for i, qi in enumerate(primes):
        qi = int(qi)
        Qi = Q // qi
        coef = (pow(Qi % qi, -1, qi) * Qi) % Q
        acc = acc + res[i].astype(object) * coef
    acc = acc % Q
    half = Q // 2
    return np.where(acc > half, acc - Q, acc)


# --------------------------------------------------------------------------
# Encoder (canonical embedding, slot j <-> zeta^(5^j))
# --------------------------------------------------------------------------
def slot_exponents(n: int) -> np.ndarray:
    e = np.empty(n // 2, dtype=np.int64)
    x = 1
    for j in range(n // 2):
        e[j] = x
        x = (x * 5) % (2 * n)
    return e


def encode_unscaled(z, n: int) -> np.ndarray:
    """Real polynomial u (float64, length n) with u(zeta^(5^j)) = z_j for j < n/2."""
    z = np.asarray(z, dtype=np.complex128)
    full = np.zeros(n // 2, dtype=np.complex128)
    full[: z.shape[0]] = z
    e = slot_exponents(n)
    vals = np.zeros(n, dtype=np.complex128)          # vals[t] = u(zeta^(2t+1))
    vals[(e - 1) // 2] = full
    vals[(2 * n - e - 1) // 2] = np.conj(full)
    a = np.fft.fft(vals) / n                         # a_k = u_k zeta^k
    k = np.arange(n)
    return (a * np.exp(-1j * np.pi * k / n)).real


def decode_coeffs(m, n: int) -> np.ndarray:
    """Slot values (complex) of a real coefficient vector m (float)."""
    m = np.asarray(m, dtype=np.float64)
    k = np.arange(n)
    a = m * np.exp(1j * np.pi * k / n)
    vals = np.fft.ifft(a) * n                         # vals[t] = m(zeta^(2t+1))
    return vals[(slot_exponents(n) - 1) // 2]


def encode(z, scale: float, n: int) -> np.ndarray:
    return rha(scale * encode_unscaled(z, n))


# --------------------------------------------------------------------------
# Keys and ciphertexts
# --------------------------------------------------------------------------
@dataclass
class Ct:
    c: np.ndarray   # [2][level+1][n] uint64, coefficient domain
    level: int


@dataclass
class SwitchKey:
    """Hybrid switching key: data[j][0] = b_j, data[j][1] = a_j over q_0..q_L, p_0..p_{alpha-1}.
    seed: when not None, every a_j comes from the seeded generator (seeded_key_a), so
    the key travels as its b part and the seed."""
    data: np.ndarray  # [beta_L][2][L+1+alpha][n]
    seed: int | None = None


@dataclass
class Keys:
    s: np.ndarray                  # ternary secret, int64 [n]
    pk: np.ndarray                 # [2][L+1][n]
    rlk: SwitchKey
    gal: dict = field(default_factory=dict)   # galois element -> SwitchKey


class Sampler:
    """Key and encryption randomness (numpy PCG64, seeded).  Only the oracle's own
    keys and encryptions use it; the CUDA path receives them as inputs."""

    def __init__(self, seed: int):
        self.rng = np.random.default_rng(seed)

    def ternary(self, n):
        return self.rng.integers(-1, 2, size=n).astype(np.int64)

    def gaussian(self, n, sigma=3.19):
        return np.rint(self.rng.normal(0.0, sigma, size=n)).astype(np.int64)

    def uniform(self, primes, n):
        return np.stack([self.rng.integers(0, int(qi), size=n, dtype=np.uint64) for qi in primes])


def galois_left(r: int, n: int) -> int:
    """Galois element of a left rotation by r slots (slot j <- slot j + r)."""
    return pow(5, r % (n // 2), 2 * n)


def galois_right(r: int, n: int) -> int:
    return galois_left((n // 2 - r % (n // 2)) % (n // 2), n)


def _brev_perm(logn: int) -> np.ndarray:
    k = np.arange(1 << logn)
    r = np.zeros_like(k)
    for b in range(logn):
        r |= ((k >> b) & 1) << (logn - 1 - b)
    return r


def seeded_key_a(P: Params, seed: int, j: int) -> np.ndarray:
    """a_j of a seeded switching key, coefficient domain over q_0..q_L, p_0..: the
    generator (SplitMix64, see the C core) gives a_j 2^64 mod q_p at evaluation index i,
    the evaluation at psi^(2 brev(i) + 1) (psi the first c^((q-1)/2n), c = 2, 3, ..., of
    order 2n); the coefficients are the negacyclic inverse transform of those values."""
    primes = P.qp(P.L)
    T = len(primes)
    ar = np.empty((T, P.n), dtype=np.uint64)
    _lib.lib().orc_seeded_key_a(int(seed) & (2**64 - 1), j, T, ptr(u64(primes)), T, P.n, ptr(ar))
    rinv = [pow(pow(2, 64, int(q)), -1, int(q)) for q in primes]
    a_eval = mul_scalar_mod(ar, rinv, primes)
    logn = P.n.bit_length() - 1
    a = np.ascontiguousarray(a_eval[:, _brev_perm(logn)])   # natural order: index m <-> psi^(2m + 1)
    # one inverse transform per prime, independent of each other: run them on threads
    # (the C core releases the interpreter lock)
    with ThreadPoolExecutor(max_workers=min(len(primes), os.cpu_count() or 1)) as ex:
        list(ex.map(lambda pq: _lib.lib().orc_nega_inverse(ptr(a[pq[0]]), P.n, int(pq[1])), enumerate(primes)))
    return a


def _switch_key(P: Params, smp: Sampler, s_all: np.ndarray, s_prime_all: np.ndarray, seed: int | None = None) -> SwitchKey:
    """Key that switches s' to s (Sec. 2.1 rotations / relinearisation); with a seed,
    the a parts come from the seeded generator."""
    primes = P.qp(P.L)
    nq = P.L + 1
    Pprod = 1
    for pk in P.p:
        Pprod *= pk
    beta = P.beta(P.L)
    data = np.empty((beta, 2, len(primes), P.n), dtype=np.uint64)
    for j in range(beta):
        lo, hi = j * P.dsize, min((j + 1) * P.dsize, nq)
        a = smp.uniform(primes, P.n) if seed is None else seeded_key_a(P, seed, j)
        e = to_residues(smp.gaussian(P.n), primes)
        b = sub_mod(e, ring_mul(a, s_all, primes), primes)
        gadget = np.zeros(len(primes), dtype=np.uint64)   # [P * E_j] mod each prime
        for t in range(lo, hi):
            gadget[t] = Pprod % primes[t]
        b = add_mod(b, mul_scalar_mod(s_prime_all, gadget, primes), primes)
        data[j, 0] = b
        data[j, 1] = a
    return SwitchKey(data, seed)


def _key_seed(seed: int, which: int) -> int:
    """Seed of one switching key's a parts (which: 1 relinearisation, else the Galois element)."""
    return (int(seed) * 0x100000001B3 + 0x51ED * int(which)) % (1 << 64)


def keygen(P: Params, seed: int, galois_elts=(), seeded: bool = True) -> Keys:
    """Secret, public key, relinearisation and Galois keys; switching keys take their
    a parts from the seeded generator unless seeded is False."""
    smp = Sampler(seed)
    s = smp.ternary(P.n)
    primes = P.qp(P.L)
    s_all = to_residues(s, primes)
    qL = P.q
    a = smp.uniform(qL, P.n)
    e = to_residues(smp.gaussian(P.n), qL)
    pk = np.stack([sub_mod(e, ring_mul(a, s_all[: P.L + 1], qL), qL), a])
    s2 = ring_mul(s_all, s_all, primes)
    ks = (lambda w: _key_seed(seed, w)) if seeded else (lambda w: None)
    rlk = _switch_key(P, smp, s_all, s2, ks(1))
    keys = Keys(s=s, pk=pk, rlk=rlk)
    for g in galois_elts:
        keys.gal[int(g)] = _switch_key(P, smp, s_all, automorphism(s_all, int(g), primes), ks(int(g)))
    return keys


def add_galois_keys(P: Params, keys: Keys, seed: int, galois_elts, seeded: bool = True) -> None:
    smp = Sampler(seed)
    primes = P.qp(P.L)
    s_all = to_residues(keys.s, primes)
    for g in galois_elts:
        g = int(g)
        if g not in keys.gal:
            keys.gal[g] = _switch_key(P, smp, s_all, automorphism(s_all, g, primes), _key_seed(seed, g) if seeded else None)


def encrypt(P: Params, keys: Keys, z, seed: int, level: int | None = None) -> Ct:
    """Secret-key encryption of slot vector z at level `level` (default L), scale Delta_level."""
    lvl = P.L if level is None else level
    smp = Sampler(seed)
    primes = P.q[: lvl + 1]
    m = to_residues(encode(z, P.scales[lvl], P.n), primes)
    a = smp.uniform(primes, P.n)
    e = to_residues(smp.gaussian(P.n), primes)
    s_res = to_residues(keys.s, primes)
    c0 = add_mod(sub_mod(e, ring_mul(a, s_res, primes), primes), m, primes)
    return Ct(np.stack([c0, a]), lvl)


def decrypt_coeffs(P: Params, keys: Keys, ct: Ct):
    primes = P.q[: ct.level + 1]
    s_res = to_residues(keys.s, primes)
    m = add_mod(ct.c[0], ring_mul(ct.c[1], s_res, primes), primes)
    return crt_centered(m, primes)


def decrypt(P: Params, keys: Keys, ct: Ct) -> np.ndarray:
    m = decrypt_coeffs(P, keys, ct).astype(np.float64) / P.scales[ct.level]
    return decode_coeffs(m, P.n).real


# --------------------------------------------------------------------------
# Homomorphic operations
# --------------------------------------------------------------------------
def mod_up(P: Params, d: np.ndarray, j: int, level: int) -> np.ndarray:
    lo, hi = j * P.dsize, min((j + 1) * P.dsize, level + 1)
    return fast_base_conv(d[lo:hi], P.q[lo:hi], P.qp(level))


def mod_down(P: Params, u: np.ndarray, level: int) -> np.ndarray:
    """(u - [u]_P) / P over Q_l, [u]_P by the centred fast conversion, so that the
    result is round(u / P) up to an error u' of mean zero (an uncentred conversion
    would bias every key switch by about (alpha - 1)/2 per coefficient)."""
    q = P.q[: level + 1]
    w = fast_base_conv_centered(u[level + 1:], P.p, q)
    Pprod = 1
    for pk in P.p:
        Pprod *= pk
    pinv = [pow(Pprod % qi, -1, qi) for qi in q]
    return mul_scalar_mod(sub_mod(u[: level + 1], w, q), pinv, q)


def base_conv_rounded(x, src, dst):
    """Basis conversion to the centred representative of x mod prod(src): the
    multiple of the product is decided by rounding sum_i y_i / s_i in IEEE double
    (see the C core); exact unless that sum lies within double rounding of a
    half-integer."""
    x = u64(x)
    out = np.empty((len(dst), x.shape[1]), dtype=np.uint64)
    _lib.lib().orc_base_conv_rounded(ptr(x), x.shape[1], ptr(u64(src)), len(src), ptr(u64(dst)), len(dst), ptr(out))
    return out


def mod_down_rescale(P: Params, u: np.ndarray, level: int) -> np.ndarray:
    """round(u / S) over Q_(l-1), S = P q_l: (u - [u]_S) / S with [u]_S the centred
    representative of u mod S from the basis {q_l, p_0 .. p_(alpha-1)} (rounded
    conversion): a key switch's ModDown and the rescale that follows it, in one
    rounding (u over Q_l P, limbs 0..l then the P limbs)."""
    q = P.q[:level]
    src_primes = [P.q[level]] + list(P.p)
    src = np.concatenate([u[level:level + 1], u[level + 1:]])
    w = base_conv_rounded(src, src_primes, q)
    S = int(P.q[level])
    for pk in P.p:
        S *= int(pk)
    sinv = [pow(S % int(qi), -1, int(qi)) for qi in q]
    return mul_scalar_mod(sub_mod(u[:level], w, q), sinv, q)


def key_switch_raw(P: Params, d: np.ndarray, key: SwitchKey, level: int, g: int | None = None):
    """Inner products u_0, u_1 over Q_l P of the lifted digits of d (automorphism g
    on the digits) with the switching key, before ModDown."""
    primes = P.qp(level)
    sel = list(range(level + 1)) + list(range(P.L + 1, P.L + 1 + P.alpha))
    beta = P.beta(level)
    digits = np.stack([mod_up(P, d, j, level) for j in range(beta)])
    if g is not None:
        digits = np.stack([automorphism(dg, g, primes) for dg in digits])
    kb = np.ascontiguousarray(key.data[:beta, 0][:, sel])
    ka = np.ascontiguousarray(key.data[:beta, 1][:, sel])
    return ring_mac(digits, kb, primes), ring_mac(digits, ka, primes)


def key_switch(P: Params, d: np.ndarray, key: SwitchKey, level: int, g: int | None = None):
    u0, u1 = key_switch_raw(P, d, key, level, g)
    return mod_down(P, u0, level), mod_down(P, u1, level)


def rescale(P: Params, ct: Ct) -> Ct:
    lvl = ct.level
    assert lvl >= 1
    ql = int(P.q[lvl])
    q = P.q[:lvl]
    last = ct.c[:, lvl, :].astype(np.int64)
    cbar = np.where(last > (ql - 1) // 2, last - ql, last)     # centred lift
    out = np.empty((2, lvl, P.n), dtype=np.uint64)
    qinv = [pow(ql % qi, -1, qi) for qi in q]
    for c in range(2):
        lift = to_residues(cbar[c], q)
        out[c] = mul_scalar_mod(sub_mod(ct.c[c, :lvl], lift, q), qinv, q)
    return Ct(out, lvl - 1)


def add(P, x: Ct, y: Ct) -> Ct:
    assert x.level == y.level, (x.level, y.level)
    q = P.q[: x.level + 1]
    return Ct(np.stack([add_mod(x.c[i], y.c[i], q) for i in range(2)]), x.level)


def sub(P, x: Ct, y: Ct) -> Ct:
    assert x.level == y.level, (x.level, y.level)
    q = P.q[: x.level + 1]
    return Ct(np.stack([sub_mod(x.c[i], y.c[i], q) for i in range(2)]), x.level)


def neg(P, x: Ct) -> Ct:
    q = P.q[: x.level + 1]
    return Ct(np.stack([neg_mod(x.c[i], q) for i in range(2)]), x.level)


def rotate(P: Params, keys: Keys, x: Ct, r: int) -> Ct:
    """Left rotation by r slots; the automorphism is applied to the lifted digits."""
    r %= P.slots
    if r == 0:
        return Ct(x.c.copy(), x.level)
    g = galois_left(r, P.n)
    q = P.q[: x.level + 1]
    k0, k1 = key_switch(P, x.c[1], keys.gal[g], x.level, g)
    c0 = add_mod(automorphism(x.c[0], g, q), k0, q)
    return Ct(np.stack([c0, k1]), x.level)


def rotate_sum(P: Params, keys: Keys, x: Ct, rs) -> Ct:
    """x + sum_k (x << r_k) for nonzero rotations r_k with one ModDown for the sum:
    the inner products of x's lifted digits (automorphism g_k on the digits, the key
    of g_k) are added over Q_l P first, then brought down once; c0 takes x's c0 and
    its automorphic images, c1 takes x's c1.  Equal to adding the separate rotations
    up to the ModDown's rounding (one rounding instead of one per rotation)."""
    q = P.q[: x.level + 1]
    primes = P.qp(x.level)
    U0 = U1 = None
    c0 = x.c[0].copy()
    for r in rs:
        g = galois_left(r % P.slots, P.n)
        assert g != 1, "rotate_sum takes nonzero rotations"
        u0, u1 = key_switch_raw(P, x.c[1], keys.gal[g], x.level, g)
        U0 = u0 if U0 is None else add_mod(U0, u0, primes)
        U1 = u1 if U1 is None else add_mod(U1, u1, primes)
        c0 = add_mod(c0, automorphism(x.c[0], g, q), q)
    c0 = add_mod(c0, mod_down(P, U0, x.level), q)
    c1 = add_mod(x.c[1], mod_down(P, U1, x.level), q)
    return Ct(np.stack([c0, c1]), x.level)


def mul(P: Params, keys: Keys, x: Ct, y: Ct) -> Ct:
    assert x.level == y.level, (x.level, y.level)
    lvl = x.level
    q = P.q[: lvl + 1]
    d0 = ring_mul(x.c[0], y.c[0], q)
    d1 = ring_mac(np.stack([x.c[0], x.c[1]]), np.stack([y.c[1], y.c[0]]), q)
    d2 = ring_mul(x.c[1], y.c[1], q)
    # relinearisation and rescale in one rounding: (P d_i + u_i) / (P q_l)
    u0, u1 = key_switch_raw(P, d2, keys.rlk, lvl)
    Pprod = 1
    for pk in P.p:
        Pprod *= int(pk)
    pm = [Pprod % int(qi) for qi in q]
    out = []
    for d, u in ((d0, u0), (d1, u1)):
        U = u.copy()
        U[: lvl + 1] = add_mod(u[: lvl + 1], mul_scalar_mod(d, pm, q), q)
        out.append(mod_down_rescale(P, U, lvl))
    return Ct(np.stack(out), lvl - 1)


def scalar_scale(P: Params, level: int) -> float:
    """Scale s at which a factor is encoded so that, after one rescale, the product
    sits at the canonical scale of level-1."""
    return (P.scales[level - 1] * float(P.q[level])) / P.scales[level]


def mul_scalar(P: Params, x: Ct, c: float) -> Ct:
    lvl = x.level
    q = P.q[: lvl + 1]
    K = rha_scalar(float(c) * scalar_scale(P, lvl))
    consts = [K % qi for qi in q]
    out = np.stack([mul_scalar_mod(x.c[i], consts, q) for i in range(2)])
    return rescale(P, Ct(out, lvl))


def plain_at(P: Params, u: np.ndarray, level: int) -> np.ndarray:
    """Residues of the plaintext with unscaled coefficients u, encoded for a product at `level`."""
    return to_residues(rha(scalar_scale(P, level) * np.asarray(u, dtype=np.float64)), P.q[: level + 1])


def mul_plain(P: Params, x: Ct, u: np.ndarray) -> Ct:
    lvl = x.level
    q = P.q[: lvl + 1]
    m = plain_at(P, u, lvl)
    out = np.stack([ring_mul(x.c[i], m, q) for i in range(2)])
    return rescale(P, Ct(out, lvl))


def add_plain(P: Params, x: Ct, u: np.ndarray) -> Ct:
    """Add the plaintext with unscaled coefficients u, encoded at the ciphertext's
    canonical scale Delta_l (rounded half away from zero), to c0.  No level is used."""
    lvl = x.level
    q = P.q[: lvl + 1]
    m = to_residues(rha(P.scales[lvl] * np.asarray(u, dtype=np.float64)), q)
    return Ct(np.stack([add_mod(x.c[0], m, q), x.c[1].copy()]), lvl)


def lincomb(P: Params, xs, cs) -> Ct:
    """sum_i c_i x_i for ciphertexts at one level l: each x_i is multiplied by the
    integer rha(c_i * s_l) (s_l as for a scalar product), the products are summed
    exactly, and the sum is rescaled once (result at level l-1)."""
    lvl = xs[0].level
    assert all(x.level == lvl for x in xs)
    q = P.q[: lvl + 1]
    s = scalar_scale(P, lvl)
    acc = np.zeros((2, lvl + 1, P.n), dtype=np.uint64)
    for x, c in zip(xs, cs):
        K = rha_scalar(float(c) * s)
        consts = [K % qi for qi in q]
        for i in range(2):
            acc[i] = add_mod(acc[i], mul_scalar_mod(x.c[i], consts, q), q)
    return rescale(P, Ct(acc, lvl))


def add_const(P: Params, x: Ct, c: float) -> Ct:
    lvl = x.level
    q = P.q[: lvl + 1]
    K = rha_scalar(float(c) * P.scales[lvl])
    out = x.c.copy()
    for i, qi in enumerate(q):
        out[0, i, 0] = (int(out[0, i, 0]) + K % qi) % qi
    return Ct(out, lvl)


def level_down(P: Params, x: Ct, target: int) -> Ct:
    while x.level > target:
        x = mul_scalar(P, x, 1.0)
    return x
