"""The value of an order statistic from the all-ties mask (Sec. 3.2): <O, V> divided
by the mask's L1 norm with Goldschmidt's iteration.

* CPU pins: the iteration's product against 1/x on a dense grid of x in [1/N, 1]
  (relative error at most 2^-10, the bound the iteration count is chosen for); the
  value in the noiseless model against numpy's min and max, with ties; zero when no
  element has rank k.
* GPU: with the oracle's keys, input and encodings imported, the CUDA circuit returns
  the oracle's ciphertext bit for bit (n = 2^11, 36 limbs, a test ring).
"""
import numpy as np
import pytest

from oracle import ckks, circuits as C
from tests import helpers


@pytest.mark.parametrize("N", [2, 8, 32, 128])
def test_goldschmidt_inverse_within_its_bound(N):
    d = C.goldschmidt_iterations(N)
    assert (1 - 1 / N) ** (2 ** (d + 1)) <= 2.0 ** -10 < (1 - 1 / N) ** (2 ** d)
    x = np.linspace(1.0 / N, 1.0, 4097)
    B = C.PlainSlots(x.size, 2 + d)
    inv = B.values(C.inverse_goldschmidt(B, B.fresh(x), d))
    assert np.max(np.abs(inv * x - 1.0)) <= 2.0 ** -10
    assert C.goldschmidt_iterations(8) == 5 and C.goldschmidt_iterations(128) == 9


@pytest.mark.parametrize("name", ["ties", "distinct"])
def test_value_all_is_the_min_and_max(name):
    v = {"ties": np.array([3, 1, 3, 1, 2, 1, 3, 2]) / 4.0,
         "distinct": np.array([0.5, 0.125, 0.875, 0.25, 0.0625, 0.625, 0.375, 0.75])}[name]
    for k, want in ((1, v.min()), (8, v.max())):
        B = C.PlainSlots(256, 60)
        got = B.values(C.order_value_all(B, B.fresh(v), 8, k, 4, 2))
        assert abs(got[0] - want) < 2e-3
        assert np.max(np.abs(got[1:8])) < 1e-9          # SumC's mask: only slot 0 of row 0


def test_value_all_is_zero_without_rank_k():
    """Fractional ranks of [a, a, a, b] are 2, 2, 2, 4: no element of rank 3 (the window
    is zero at the integers around k), so the value is zero.  (k = 1 would take Cmp_G,
    which gives every minimum rank 1.)"""
    v = np.array([0.25, 0.25, 0.25, 0.5])
    assert list(C.brute_fractional_rank(v)) == [2, 2, 2, 4]
    for k in (3,):
        B = C.PlainSlots(64, 60)
        got = B.values(C.order_value_all(B, B.fresh(v), 4, k, 4, 2))
        assert abs(got[0]) < 1e-3, k


@pytest.mark.gpu
def test_value_all_bit_exact():
    P = helpers.oracle_params("deep")
    N = 8
    keys = ckks.keygen(P, 81, helpers.galois_elts(P, helpers.rotation_set(N)))
    ctx = helpers.gpu_context("deep")
    try:
        helpers.import_keys(ctx, keys)
        helpers.import_encodings(ctx, P, N, kinds=helpers.ALL_MASKS)
        ctx.indicator_import(N, C.sinc2_window_coeffs(N))
        v = np.array([3, 1, 3, 1, 2, 1, 3, 2]) / 4.0
        ct = ckks.encrypt(P, keys, v, 82)
        B = C.OracleCkks(P, keys)
        for k, want in ((1, v.min()), (N, v.max())):
            ref = C.order_value_all(B, ct, N, k, 2, 1)
            g = ctx.order_value_all(ctx.ct_import(ct.c, ct.level, N=N), k)
            assert g.level == ref.level
            assert np.array_equal(g.export(), ref.c)
            assert abs(ctx.decrypt(g)[0] - want) < 0.02
    finally:
        ctx.close()
