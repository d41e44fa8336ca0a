"""The library's 64-bit modular arithmetic (csrc/modarith.cuh), compiled for the host
with g++, against Python's integers: Shoup's product, Montgomery's reduction, and
their forms for primes k 2^32 + 1 (one or two 32-bit products by q), which must give
the same words as the general forms."""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2412_15126_gb300", "csrc")

PROGRAM = r"""
#define __host__
#define __device__
#define __forceinline__ inline
#include "modarith.cuh"
#include <cstdio>
int main() {
    unsigned long long q, a, w, lo, hi;
    while (scanf("%llu %llu %llu %llu %llu", &q, &a, &w, &lo, &hi) == 5) {
        u64 qinv = 1;
        for (int i = 0; i < 7; i++) qinv *= 2 - q * qinv;
        const u64 wp = (u64)(((u128)w << 64) / q);
        printf("%llu %llu %llu %llu %llu %llu %llu %d\n",
               (unsigned long long)shoup_lazy(a, w, wp, q), (unsigned long long)shoup_lazy_t<true>(a, w, wp, q),
               (unsigned long long)mont_redc(lo, hi, q, qinv), (unsigned long long)mont_redc_t<true>(lo, hi, q, qinv),
               (unsigned long long)mul_q_lo_k32(a, q), (unsigned long long)mulhi_q_k32(a, q),
               (unsigned long long)umulhi64(a, q), (int)is_k32_prime(q));
    }
    return 0;
}
"""


def _is_prime(x):
    if x < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if x % p == 0:
            return x == p
    d, s = x - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        y = pow(a, d, x)
        if y in (1, x - 1):
            continue
        for _ in range(s - 1):
            y = y * y % x
            if y == x - 1:
                break
        else:
            return False
    return True


def _k32_primes():
    """Three primes k 2^32 + 1 at or below each of k = 2^13 (near 2^45), 2^18 (2^50),
    2^28 (2^60) and 2^29 - 1 (the largest below 2^61)."""
    out = []
    for k0 in (1 << 13, 1 << 18, 1 << 28, (1 << 29) - 1):
        k, found = k0, 0
        while found < 3:
            if _is_prime((k << 32) + 1):
                out.append((k << 32) + 1)
                found += 1
            k -= 1
    return out


@pytest.fixture(scope="module")
def binary(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("modarith")
    src = d / "check.cpp"
    src.write_text(PROGRAM)
    exe = d / "check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def test_k32_forms_equal_the_general_forms_and_python(binary):
    rng = random.Random(2412)
    primes = _k32_primes()
    assert len(primes) >= 10 and all(p % (1 << 32) == 1 and p < (1 << 61) for p in primes)
    lines, cases = [], []
    for q in primes:
        for _ in range(400):
            a = rng.getrandbits(64)
            w = rng.randrange(q)
            lo, hi = rng.getrandbits(64), rng.randrange(q)
            cases.append((q, a, w, lo, hi))
            lines.append("%d %d %d %d %d" % (q, a, w, lo, hi))
    out = subprocess.run([binary], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True).stdout
    rows = out.split("\n")
    for (q, a, w, lo, hi), row in zip(cases, rows):
        sg, sk, mg, mk, mlo, mhi, hig, isk = (int(x) for x in row.split())
        assert sk == sg                                    # Shoup: the same word either way
        assert sg % q == a * w % q and sg < 2 * q          # ... a w mod q, lazily in [0, 2q)
        assert mk == mg                                    # Montgomery: the same word either way
        assert mg == (hi * 2 ** 64 + lo) * pow(2 ** 64, -1, q) % q
        assert mlo == a * q % 2 ** 64                      # low word of a q
        assert mhi == hig == a * q >> 64                   # high word of a q
        assert isk == 1


def test_general_primes_are_not_taken_for_k32(binary):
    q = (1 << 61) - 1                                      # a Mersenne prime, not k 2^32 + 1
    out = subprocess.run([binary], input="%d 5 7 11 13\n" % q, capture_output=True, text=True, check=True).stdout
    assert out.split()[-1] == "0"
