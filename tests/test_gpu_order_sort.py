"""GPU parity of the order-statistic (Alg. 4) and sorting (Alg. 5, column form)
circuits, including the Paterson-Stockmeyer evaluation of the Chebyshev indicator.

* n = 2^11, 24 limbs, N = 8 (a ring the oracle runs in seconds): with the oracle's
  keys, ciphertext, mask encodings and indicator coefficients imported, the CUDA
  circuits return the oracle's ciphertexts bit for bit.
* n = 2^16, 34 limbs, N = 128 on a 64-level grid (ties): argmin, argmax and sort on
  the library's own keys decrypt to the brute-force answers.
"""
import numpy as np
import pytest

from oracle import ckks, circuits as C
from paper_2412_15126_gb300 import inputs
from tests import helpers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ord_setup():
    from paper_2412_15126_gb300 import rankfhe
    P = helpers.oracle_params("ord")
    N = 8
    keys = ckks.keygen(P, 31, helpers.galois_elts(P, helpers.rotation_set(N)))
    ctx = helpers.gpu_context("ord")
    helpers.import_keys(ctx, keys)
    helpers.import_encodings(ctx, P, N, kinds=helpers.ALL_MASKS)
    ctx.indicator_import(N, C.sinc2_window_coeffs(N))
    yield P, keys, ctx, rankfhe
    ctx.close()


VECS = {
    "ties": np.array([3, 1, 3, 0, 2, 1, 3, 2]) / 4.0,
    "distinct": np.array([0.5, 0.125, 0.875, 0.25, 0.0, 0.625, 0.375, 0.75]),
}


@pytest.mark.parametrize("name", list(VECS))
def test_argmin_first_bit_exact(ord_setup, name):
    P, keys, ctx, rk = ord_setup
    v = VECS[name]
    ct = ckks.encrypt(P, keys, v, 3)
    ref = C.order_statistic(C.OracleCkks(P, keys), ct, 8, 1, 2, 1)
    g = ctx.order_stat(ctx.ct_import(ct.c, ct.level, N=8), 1, rk.TIES_FIRST)
    assert g.level == ref.level
    assert np.array_equal(g.export(), ref.c)
    o = ctx.decrypt(g)
    first = np.zeros(8)
    first[int(np.argmin(v))] = 1
    assert np.max(np.abs(o - first)) < 0.01


def test_argmax_all_and_median_rank_bit_exact(ord_setup):
    P, keys, ctx, rk = ord_setup
    v = VECS["ties"]
    ct = ckks.encrypt(P, keys, v, 4)
    B = C.OracleCkks(P, keys)
    ref = C.order_statistic(B, ct, 8, 8, 2, 1, ties="all")
    g = ctx.order_stat(ctx.ct_import(ct.c, ct.level, N=8), 8, rk.TIES_ALL)
    assert np.array_equal(g.export(), ref.c)
    assert np.max(np.abs(ctx.decrypt(g) - (v == v.max()))) < 0.01
    ref = C.order_statistic(B, ct, 8, 4, 2, 1)
    g = ctx.order_stat(ctx.ct_import(ct.c, ct.level, N=8), 4, rk.TIES_FIRST)
    assert np.array_equal(g.export(), ref.c)


@pytest.mark.parametrize("name", list(VECS))
def test_sort_bit_exact(ord_setup, name):
    P, keys, ctx, rk = ord_setup
    v = VECS[name]
    ct = ckks.encrypt(P, keys, v, 5)
    ref = C.sort(C.OracleCkks(P, keys), ct, 8, 2, 1)
    g = ctx.sort(ctx.ct_import(ct.c, ct.level, N=8))
    assert g.level == ref.level
    assert np.array_equal(g.export(), ref.c)
    assert np.max(np.abs(ctx.decrypt(g) - np.sort(v))) < 0.01


@pytest.fixture(scope="module")
def cfg3():
    ctx = helpers.gpu_context("cfg3")
    ctx.keygen(77, 128)
    yield ctx
    ctx.close()


@pytest.mark.parametrize("seed", [1, 2])
def test_cfg3_argmin_argmax_sort_n128(cfg3, seed):
    from paper_2412_15126_gb300 import rankfhe as rk
    ctx = cfg3
    v = inputs.grid_vector(128, 64, seed)
    ct = ctx.encrypt(v, N=128)
    o = ctx.decrypt(ctx.order_stat(ct, 1, rk.TIES_FIRST))
    first = np.zeros(128)
    first[int(np.argmin(v))] = 1
    assert np.max(np.abs(o - first)) < 0.01
    o = ctx.decrypt(ctx.order_stat(ct, 128, rk.TIES_ALL))
    assert np.max(np.abs(o - (v == v.max()))) < 0.01
    s = ctx.decrypt(ctx.sort(ct))
    assert np.max(np.abs(s - np.sort(v))) < 0.01


@pytest.mark.parametrize("name", list(VECS))
def test_order_value_and_median_bit_exact(ord_setup, name):
    P, keys, ctx, rk = ord_setup
    v = VECS[name]
    ct = ckks.encrypt(P, keys, v, 6)
    B = C.OracleCkks(P, keys)
    ref = C.order_value(B, ct, 8, 3, 2, 1)
    g = ctx.order_value(ctx.ct_import(ct.c, ct.level, N=8), 3)
    assert g.level == ref.level
    assert np.array_equal(g.export(), ref.c)
    assert abs(ctx.decrypt(g)[0] - np.sort(v)[2]) < 0.01
    ref = C.median(B, ct, 8, 2, 1)
    g = ctx.median(ctx.ct_import(ct.c, ct.level, N=8))
    assert np.array_equal(g.export(), ref.c)
    assert abs(ctx.decrypt(g)[0] - np.median(v)) < 0.01


@pytest.mark.parametrize("seed", [3])
def test_cfg3_median_n128(cfg3, seed):
    ctx = cfg3
    v = inputs.grid_vector(128, 64, seed)
    m = ctx.decrypt(ctx.median(ctx.encrypt(v, N=128)))
    assert abs(m[0] - np.median(v)) < 0.01
