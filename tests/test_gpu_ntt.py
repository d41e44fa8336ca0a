"""GPU parity of the raw NTT kernels on device buffers: inverse(forward(x)) = x bit
for bit, and forward(x)[i] = x(psi^(2 brev(i) + 1)) mod q, with psi the first
c^((q-1)/2n), c = 2, 3, ..., of multiplicative order 2n (checked by direct
polynomial evaluation with Python integers on sampled indices)."""
import numpy as np
import pytest

from tests import helpers

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _psi(q, n):
    c = 2
    while True:
        w = pow(c, (q - 1) // (2 * n), q)
        if pow(w, n, q) == q - 1:
            return w
        c += 1


def _brev(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2)


def _horner(coeffs, x, q):
    acc = 0
    for c in reversed(coeffs):
        acc = (acc * x + c) % q
    return acc


@pytest.mark.parametrize("name", ["small", "cfg1", "cfg2", "ring17"])
def test_ntt_forward_inverse(name):
    ctx = helpers.gpu_context(name)
    primes = ctx.moduli()
    n = ctx.n
    logn = n.bit_length() - 1
    rng = np.random.default_rng(1)
    limbs = len(primes)
    x = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in primes])
    x[:, 0] = np.array(primes, dtype=np.uint64) - 1          # boundary residues
    x[:, 1] = 0
    dev = torch.from_numpy(x.view(np.int64).copy()).cuda()
    torch.cuda.synchronize()
    ctx.ntt_forward(dev.data_ptr(), limbs, 0)
    ctx.sync()
    X = dev.cpu().numpy().view(np.uint64)
    assert np.all(X < np.array(primes, dtype=np.uint64)[:, None])
    for t in (0, limbs // 2, limbs - 1):
        q = primes[t]
        psi = _psi(q, n)
        coeffs = [int(v) for v in x[t]]
        for i in (0, 1, 7, n // 2 + 3, n - 1):
            assert int(X[t, i]) == _horner(coeffs, pow(psi, 2 * _brev(i, logn) + 1, q), q)
    ctx.ntt_inverse(dev.data_ptr(), limbs, 0)
    ctx.sync()
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), x)
    ctx.close()


def test_ring17_rotation_and_product_bit_exact():
    """n = 2^17 (2^9-point row passes): one rotation and one product equal the
    oracle's bit for bit."""
    from oracle import ckks
    from paper_2412_15126_gb300 import inputs
    P = helpers.oracle_params("ring17")
    keys = ckks.keygen(P, 17, helpers.galois_elts(P, [-256]))
    ctx = helpers.gpu_context("ring17")
    try:
        helpers.import_keys(ctx, keys)
        ct = ckks.encrypt(P, keys, inputs.gap_vector(256, 2.0 ** -9, 17), 17)
        g = ctx.ct_import(ct.c, ct.level, N=256)
        assert np.array_equal(ctx.rotate(g, -256).export(), ckks.rotate(P, keys, ct, -256).c)
        assert np.array_equal(ctx.mul(g, g).export(), ckks.mul(P, keys, ct, ct).c)
    finally:
        ctx.close()
