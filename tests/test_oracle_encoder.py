"""Pins for the oracle's canonical-embedding encoder (Sec. 2.1: n/2 complex slots):
direct evaluation of the polynomial at the slot roots, the closed form of a
constant, and round trips."""
import numpy as np
import pytest

from oracle import ckks


@pytest.mark.parametrize("log_n", [3, 4, 6])
def test_encode_matches_direct_evaluation(log_n):
    n = 1 << log_n
    rng = np.random.default_rng(log_n)
    z = rng.uniform(-1, 1, n // 2)
    u = ckks.encode_unscaled(z, n)
    zeta = np.exp(1j * np.pi / n)
    for j in range(n // 2):
        root = zeta ** pow(5, j, 2 * n)
        val = sum(u[k] * root ** k for k in range(n))
        assert abs(val - z[j]) < 1e-12
    # decode is the same evaluation
    assert np.allclose(ckks.decode_coeffs(u, n), z, atol=1e-12)


def test_constant_encodes_to_constant_polynomial():
    n = 1 << 12
    u = ckks.encode_unscaled(np.full(n // 2, 0.375), n)
    assert abs(u[0] - 0.375) < 1e-14
    assert np.max(np.abs(u[1:])) < 1e-14


def test_scaled_round_trip():
    n = 1 << 13
    rng = np.random.default_rng(1)
    z = rng.uniform(0, 1, 300)
    m = ckks.encode(z, 2.0 ** 40, n)
    back = ckks.decode_coeffs(m.astype(np.float64) / 2.0 ** 40, n).real
    assert np.max(np.abs(back[:300] - z)) < 2.0 ** -30
    assert np.max(np.abs(back[300:])) < 2.0 ** -30
