"""GPU: the serving loop (continuous batching on a worker thread).

* A mix of rank, order-statistic, sort and blocked-rank requests returns, for every
  request, exactly the ciphertext the direct call returns for it alone.
* A request that cannot be evaluated reports its error through rk_server_wait and
  does not stop the server.
"""
import numpy as np
import pytest

from paper_2412_15126_gb300 import inputs, rankfhe
from tests import helpers

pytestmark = pytest.mark.gpu


def test_server_mix_identical_to_alone():
    ctx = helpers.gpu_context("ord")
    try:
        ctx.keygen(91, 8)
        vs = [inputs.grid_vector(8, 16, 700 + i) for i in range(9)]
        cts = [ctx.encrypt(v, N=8) for v in vs]
        blocks = ctx.stack([ctx.encrypt(inputs.gap_vector(8, 0.05, 800 + b), N=8) for b in range(3)])
        reqs = []
        for i, ct in enumerate(cts):
            if i % 3 == 0:
                reqs.append((rankfhe.OP_RANK, ct, 0, rankfhe.TIES_CORRECT))
            elif i % 3 == 1:
                reqs.append((rankfhe.OP_ORDER_STAT, ct, 1, rankfhe.TIES_FIRST))
            else:
                reqs.append((rankfhe.OP_SORT, ct, 0, 0))
        reqs.append((rankfhe.OP_RANK, cts[1], 0, 0))
        reqs.append((rankfhe.OP_RANK_BLOCKED, blocks, 0, 0))
        ctx.server_start(8 << 30, 16)
        tickets = [ctx.server_submit(op, ct, arg, flags) for op, ct, arg, flags in reqs]
        outs = [ctx.server_wait(t) for t in tickets]
        stats = ctx.server_stats()
        lat = ctx.server_latencies()
        ctx.server_stop()
        assert len(lat) == len(reqs) and min(lat) > 0
        assert stats["finished"] == len(reqs)
        assert stats["p99_s"] >= stats["p50_s"] > 0
        for (op, ct, arg, flags), got in zip(reqs, outs):
            if op == rankfhe.OP_RANK:
                ref = ctx.rank(ct, flags)
            elif op == rankfhe.OP_ORDER_STAT:
                ref = ctx.order_stat(ct, arg, flags)
            elif op == rankfhe.OP_SORT:
                ref = ctx.sort(ct, flags)
            else:
                parts = ctx.unstack(got)
                refs = ctx.rank_blocked(ctx.unstack(ct))
                for a, b in zip(parts, refs):
                    assert np.array_equal(a.export(), b.export())
                continue
            assert np.array_equal(got.export(), ref.export())
    finally:
        ctx.close()


def test_server_reports_request_errors():
    ctx = helpers.gpu_context("ord")
    try:
        ctx.keygen(5, 8)
        low = ctx.encrypt(inputs.gap_vector(8, 0.05, 1), N=8)
        while low.level > 1:
            low = ctx.mul_scalar(low, 1.0)
        ok = ctx.encrypt(inputs.gap_vector(4, 0.05, 2), N=4)
        ctx.server_start(1 << 30, 4)
        bad = ctx.server_submit(rankfhe.OP_RANK, low)
        good = ctx.server_submit(rankfhe.OP_RANK, ok)
        with pytest.raises(rankfhe.RkError):
            ctx.server_wait(bad)
        assert ctx.server_wait(good) is not None
        with pytest.raises(rankfhe.RkError):
            ctx.server_wait(good)                  # collected once
        ctx.server_stop()
    finally:
        ctx.close()
