"""The replicated (N > 1) bench path on CPU: two gloo ranks.  Each replica ranks its
own seeded vectors and the job's time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2412_15126_gb300 import inputs
        t = bench.max_over_ranks(0.5 + rank, world, device="cpu")
        v = inputs.gap_vector(128, 2.0 ** -9, bench.replica_seed(rank, 0))
        out.put((rank, t, v.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_distinct_inputs():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (t, v)) for r, t, v in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 1.5
    assert not np.array_equal(res[0][1], res[1][1])


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
