"""GPU: ranks with the Chebyshev-approximated comparison (Sec. 2.2).

* n = 2^11, 24 limbs, N = 8, 64 coefficients (depth 7): with the oracle's keys,
  ciphertext, masks and comparator coefficients imported, the rank ciphertext equals
  the oracle's bit for bit.
* n = 2^16, 28 limbs, N = 128, 512 coefficients (depth 10): the decrypted ranks match
  the noiseless model of the same circuit (the error is the approximation's, Fig. 6).
"""
import numpy as np
import pytest

from oracle import ckks, circuits as C
from paper_2412_15126_gb300 import inputs, rankfhe
from tests import helpers

pytestmark = pytest.mark.gpu


def test_cheb_rank_bit_exact_small():
    log_n, n_limbs, log_q0, log_scale, alpha, log_sp, dsize, _, _ = helpers.CONFIGS["ord"]
    P = ckks.gen_params(log_n, n_limbs, log_q0, log_scale, alpha, log_sp, dsize)
    keys = ckks.keygen(P, 51, helpers.galois_elts(P, helpers.rotation_set(8)))
    cc = C.ChebCmp(64)
    ctx = rankfhe.Context(log_n, n_limbs, alpha, dsize, log_scale, log_q0, log_sp, 0, 0, cmp_cheb=64)
    try:
        helpers.import_keys(ctx, keys)
        helpers.import_encodings(ctx, P, 8)
        ctx.comparator_import(cc.coeffs)
        v = np.array([0.5, 0.125, 0.875, 0.25, 0.0, 0.625, 0.375, 0.75])
        ct = ckks.encrypt(P, keys, v, 7)
        ref = C.rank(C.OracleCkks(P, keys), ct, 8, cc, 0)
        got = ctx.rank(ctx.ct_import(ct.c, ct.level, N=8))
        assert got.level == ref.level
        assert np.array_equal(got.export(), ref.c)
    finally:
        ctx.close()


def test_cheb_rank_n128_matches_noiseless_model():
    ctx = rankfhe.Context(16, 28, 3, 3, 45, 60, 61, 0, 0, cmp_cheb=512)
    try:
        ctx.keygen(52, 128)
        rng = np.random.default_rng(8)
        for _ in range(2):
            v = rng.uniform(0, 1, 128)
            R = ctx.decrypt(ctx.rank(ctx.encrypt(v, N=128)))
            B = C.PlainSlots(2 * 128 * 128, 40)
            Rp = B.values(C.rank(B, B.fresh(v), 128, C.ChebCmp(512), 0))[:128]
            assert np.max(np.abs(R - Rp)) < 1e-3
            assert np.mean(np.abs(R - C.brute_fractional_rank(v))) < 0.35   # Fig. 6: 0.22 at depth 10
    finally:
        ctx.close()
