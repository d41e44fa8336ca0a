"""GPU: host-side failures surface as status codes and leave the context usable (no
test faults, traps or hangs a GPU): malformed and truncated key-set blobs, key
blobs of other parameters, ciphertext imports with bad metadata, collecting
unknown tickets, submitting to a stopped server."""
import numpy as np
import pytest

from paper_2412_15126_gb300 import inputs, rankfhe
from tests import helpers

pytestmark = pytest.mark.gpu


def _status(fn):
    with pytest.raises(rankfhe.RkError) as e:
        fn()
    return e.value.status


def test_bad_key_blobs_are_refused_and_the_context_still_works():
    ctx = helpers.gpu_context("small")
    other = helpers.gpu_context("cfg1")
    try:
        ctx.keygen(5, 8)
        ct = ctx.encrypt(inputs.gap_vector(8, 0.05, 2), N=8)
        before = ctx.rotate(ct, 1).export()
        blob = ctx.keys_export()
        bad = blob.copy()
        bad[0] ^= np.uint64(1)                               # magic
        assert _status(lambda: ctx.keys_import(bad)) == rankfhe.RK_EFORMAT
        assert _status(lambda: ctx.keys_import(blob[: blob.size - 3])) == rankfhe.RK_EFORMAT   # truncated
        bad = blob.copy()
        bad[7] = np.uint64(2)                                # first record: seeded flag out of range
        assert _status(lambda: ctx.keys_import(bad)) == rankfhe.RK_EFORMAT
        other.keygen(5, 8)
        assert _status(lambda: ctx.keys_import(other.keys_export())) == rankfhe.RK_EFORMAT   # other ring
        assert np.array_equal(ctx.rotate(ct, 1).export(), before)
    finally:
        other.close()
        ctx.close()


def test_bad_ciphertext_metadata_is_refused():
    ctx = helpers.gpu_context("small")
    try:
        ctx.keygen(6, 8)
        ct = ctx.encrypt(inputs.gap_vector(8, 0.05, 3), N=8)
        c = ct.export()
        assert _status(lambda: ctx.ct_import(c, 99, N=8)) == rankfhe.RK_EINVAL     # level beyond the chain
        assert _status(lambda: ctx.ct_import(c, c.shape[1] - 1, N=8, n_real=9)) == rankfhe.RK_EINVAL
        assert _status(lambda: ctx.ct_import(c, c.shape[1] - 1, N=8, Q=0)) == rankfhe.RK_EINVAL
        g = ctx.ct_import(c, c.shape[1] - 1, N=8)
        assert np.array_equal(g.export(), c)
    finally:
        ctx.close()


def test_server_tickets_and_stop():
    ctx = helpers.gpu_context("cfg1")
    try:
        ctx.keygen(7, 8)
        ct = ctx.encrypt(inputs.gap_vector(8, 0.05, 4), N=8)
        ctx.server_start(1 << 32)
        t = ctx.server_submit(rankfhe.OP_RANK, ct)
        assert _status(lambda: ctx.server_wait(t + 12345, 0.0)) == rankfhe.RK_EINVAL   # unknown ticket
        r = ctx.server_wait(t, -1.0)
        assert r is not None
        assert _status(lambda: ctx.server_wait(t, 0.0)) == rankfhe.RK_EINVAL          # collected already
        ctx.server_stop()
        assert _status(lambda: ctx.server_submit(rankfhe.OP_RANK, ct)) == rankfhe.RK_EINVAL   # no server
        assert np.array_equal(r.export(), ctx.rank(ct).export())
    finally:
        ctx.close()
