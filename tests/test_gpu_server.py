"""GPU: the serving loop (continuous batching over concurrent execution lanes).

* A mix of rank, order-statistic, sort and blocked-rank requests returns, for every
  request, exactly the ciphertext the direct call returns for it alone (no packing
  keys: every batch is a stack).
* With the packing rotations' keys, short requests of one shape are slot-packed
  (Q per ciphertext): each decrypts to its result alone within 1e-3, and to the
  brute-force answer.
* Two lanes run batches at the same time; a budget that admits one batch's working
  set at a time keeps them to one.
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


def _packing_rotations(N, slots):
    rs, s = [], 1
    while s * N * N < slots:
        rs += [N * N * s, -N * N * s]
        s *= 2
    return rs


def test_server_packs_short_requests_within_tolerance():
    """Eleven 8-element requests of three operations on the n = 2^11 ring (16 queries a
    ciphertext): each operation's requests share packed ciphertexts; every result
    decrypts to the request's result alone within 1e-3 in its slots."""
    from oracle.circuits import brute_tie_corrected_rank
    ctx = helpers.gpu_context("ord")
    try:
        ctx.keygen(92, 8)
        ctx.keygen_rotations(_packing_rotations(8, ctx.n // 2))
        vs = [inputs.grid_vector(8, 16, 900 + i) for i in range(11)]
        cts = [ctx.encrypt(v, N=8) for v in vs]
        ops = [(rankfhe.OP_RANK, 0, rankfhe.TIES_CORRECT), (rankfhe.OP_ORDER_STAT, 1, rankfhe.TIES_FIRST),
               (rankfhe.OP_SORT, 0, 0)]
        reqs = [(ops[i % 3], ct, v) for i, (ct, v) in enumerate(zip(cts, vs))]
        ctx.server_start(8 << 30, 16)
        tickets = [ctx.server_submit(op, ct, arg, flags) for (op, arg, flags), ct, _ in reqs]
        outs = [ctx.server_wait(t) for t in tickets]
        lanes = ctx.server_stats_lanes()
        ctx.server_stop()
        assert lanes["packed_requests"] >= 6
        for ((op, arg, flags), ct, v), got in zip(reqs, outs):
            if op == rankfhe.OP_RANK:
                alone, want = ctx.rank(ct, flags), brute_tie_corrected_rank(v)
            elif op == rankfhe.OP_ORDER_STAT:
                alone, want = ctx.order_stat(ct, arg, flags), np.eye(8)[int(np.argmin(v))]
            else:
                alone, want = ctx.sort(ct), np.sort(v)
            g, a = ctx.decrypt(got), ctx.decrypt(alone)
            assert np.max(np.abs(g - a)) < 1e-3, op
            assert np.max(np.abs(g - want)) < (0.25 if op == rankfhe.OP_RANK else 0.01), op
    finally:
        ctx.close()


def test_server_lanes_overlap_and_budget_admission():
    """Two lanes: requests of different shapes run on both lanes at once; a budget
    smaller than one batch's working set admits one batch at a time."""
    ctx = helpers.gpu_context("ord")
    try:
        ctx.keygen(93, 8)
        cts = [ctx.encrypt(inputs.gap_vector(N, 0.05, 950 + i), N=N) for i, N in enumerate([8, 4, 2, 8, 4, 2])]
        ops = [rankfhe.OP_RANK, rankfhe.OP_SORT]
        busy = {}
        for budget in (8 << 30, 1):
            ctx.set_option(rankfhe.OPT_SERVER_LANES, 2)
            ctx.server_start(budget, 1)
            tickets = [ctx.server_submit(ops[i % 2], ct) for i, ct in enumerate(cts)]
            outs = [ctx.server_wait(t) for t in tickets]
            busy[budget] = ctx.server_stats_lanes()
            ctx.server_stop()
            for i, (ct, got) in enumerate(zip(cts, outs)):
                ref = ctx.rank(ct) if i % 2 == 0 else ctx.sort(ct)
                assert np.array_equal(got.export(), ref.export())
        assert busy[8 << 30]["lanes"] == 2 and busy[8 << 30]["max_lanes_busy"] == 2
        assert busy[1]["max_lanes_busy"] == 1
    finally:
        ctx.close()
