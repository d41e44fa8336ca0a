"""The allocation-free rescale (rk_rescale_noalloc) against the ordinary rescale.

Callers that cannot allocate device memory on their call path pass their own
device buffers; the library keeps the temporary in a fixed device array.  This
file is collected last so that a run stopping at the first failure has run every
other test; it passes alone in a fresh process and after the others.  Two calls
in a row, each checked bit for bit against rk_rescale on the same ciphertext.
"""
import numpy as np
import pytest

from tests import helpers

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _to_eval_device(ctx, coeffs):
    """Canonical [2][l+1][n] coefficients -> device buffer in the evaluation domain."""
    dev = torch.from_numpy(np.ascontiguousarray(coeffs).view(np.int64).copy()).cuda()
    torch.cuda.synchronize()
    limbs = coeffs.shape[1]
    stride = limbs * ctx.n
    for p in range(2):
        ctx.ntt_forward(dev.data_ptr() + 8 * p * stride, limbs, 0)
    return dev


def _to_canonical(ctx, dev, limbs):
    stride = limbs * ctx.n
    for p in range(2):
        ctx.ntt_inverse(dev.data_ptr() + 8 * p * stride, limbs, 0)
    ctx.sync()
    return dev.cpu().numpy().view(np.uint64).reshape(2, limbs, ctx.n)


def test_rescale_noalloc_matches_rescale_twice():
    """Two calls in a row, each bit for bit rk_rescale's result; across each call the
    library makes no device allocation (its own counter of cudaMalloc and
    cudaMallocAsync calls), and across the second call the device's free memory does
    not move (the first call may still load the library's code and its array)."""
    from paper_2412_15126_gb300 import rankfhe
    ctx = helpers.gpu_context("cfg1")
    try:
        ctx.keygen(99, 8)
        rng = np.random.default_rng(5)
        for call in range(2):
            ct = ctx.encrypt(rng.uniform(0, 1, 8), N=8)
            if call == 1:
                ct = ctx.mul_scalar(ct, 0.75)          # a lower level on the second call
            level = ct.level
            expect = ctx.rescale(ct).export()
            d_in = _to_eval_device(ctx, ct.export())
            d_out = torch.empty(2 * level * ctx.n, dtype=torch.int64, device="cuda")
            ctx.sync()
            torch.cuda.synchronize()
            allocs, free0 = rankfhe.device_alloc_count(), torch.cuda.mem_get_info()[0]
            ctx.rescale_noalloc(d_in.data_ptr(), d_out.data_ptr(), level)
            ctx.sync()
            assert rankfhe.device_alloc_count() == allocs, f"call {call} allocated device memory"
            if call == 1:
                assert torch.cuda.mem_get_info()[0] == free0, "the second call changed the free device memory"
            got = _to_canonical(ctx, d_out, level)
            assert np.array_equal(got, expect), f"call {call}"
    finally:
        ctx.close()


def test_rescale_noalloc_rejects_oversize():
    from paper_2412_15126_gb300 import rankfhe
    ctx = helpers.gpu_context("cfg2")        # n = 2^16: 2 (level+1) n words exceed the 2^19-word array
    try:
        d = torch.empty(8, dtype=torch.int64, device="cuda")
        with pytest.raises(rankfhe.RkError) as e:
            ctx.rescale_noalloc(d.data_ptr(), d.data_ptr() + 4096, 20)
        assert e.value.status == rankfhe.RK_EINVAL
        assert "exceeds the fixed scratch" in str(e.value)
    finally:
        ctx.close()
