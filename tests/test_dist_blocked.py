"""The blocked rank divided between processes (the block pairs of Alg. 7 across
devices, one all-gather of the per-block partial sums), on CPU: two gloo ranks with
the oracle's RNS-CKKS as the evaluator.  Every rank's assembled ranks equal the
oracle's single-process rank_blocked bit for bit.  The CUDA evaluator runs the same
partition on one GPU in tests/test_gpu_blocked.py; several GPUs are unmeasured here.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2412_15126_gb300 import blocked_dist  # noqa: E402


class OracleEvaluator:
    """Alg. 7 split as the library splits it (rk_rank_blocked_partial / _finish), on
    the oracle: comparisons of the listed pairs and per-block partial sums, then
    R_i = TransC(SumC(i - B_i)) + SumR(A_i) + 1/2 (Eq. 3)."""

    def __init__(self, P, keys, Bsz, dg, df):
        from oracle import circuits as C
        self.C = C
        self.P, self.keys, self.Bsz, self.dg, self.df = P, keys, Bsz, dg, df
        self.B = C.OracleCkks(P, keys)

    def partial(self, blocks, pairs):
        from oracle import ckks
        C, B = self.C, self.B
        forms = [C.row_col_forms(B, V, self.Bsz) for V in blocks]
        L = len(blocks)
        A, Bs = [None] * L, [None] * L
        for i, j in pairs:
            Cij = C.cmp(B, B.sub(forms[i][0], forms[j][1]), self.dg, self.df)
            A[i] = Cij if A[i] is None else B.add(A[i], Cij)
            if j > i:
                Bs[j] = Cij if Bs[j] is None else B.add(Bs[j], Cij)
        lvl = forms[0][1].level - C.cmp_levels(self.dg, self.df)
        zero = ckks.Ct(np.zeros((2, lvl + 1, self.P.n), dtype=np.uint64), lvl)
        return [a if a is not None else zero for a in A], [b if b is not None else zero for b in Bs]

    def finish(self, A, Bs):
        C, B, Bsz = self.C, self.B, self.Bsz
        out = []
        for i in range(len(A)):
            S = C.sum_r(B, A[i], Bsz)
            if i > 0:
                T = C.trans_c(B, C.sum_c(B, B.add_const(B.neg(Bs[i]), float(i)), Bsz), Bsz)
                R = B.add(B.level_down(S, B.level(T)), T)
            else:
                R = B.level_down(S, B.level(S) - 1)
            out.append(B.add_const(R, 0.5))
        return out

    def add(self, a, b):
        return self.B.add(a, b)

    def export(self, ct):
        return ct.c

    def import_(self, arr, like):
        from oracle import ckks
        return ckks.Ct(np.array(arr, dtype=np.uint64), like.level)


def _setup():
    from oracle import ckks
    from paper_2412_15126_gb300 import inputs
    from tests import helpers
    P = helpers.oracle_params("ord")
    keys = ckks.keygen(P, 61, helpers.galois_elts(P, helpers.rotation_set(8)))
    v = inputs.gap_vector(24, 0.04, 62)
    blocks = [ckks.encrypt(P, keys, v[8 * i: 8 * i + 8], 63 + i) for i in range(3)]
    return P, keys, v, blocks


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import circuits as C, ckks
        P, keys, v, blocks = _setup()
        ev = OracleEvaluator(P, keys, 8, 2, 1)
        got = blocked_dist.blocked_rank_distributed(ev, blocks, rank, world)
        ref = C.rank_blocked(C.OracleCkks(P, keys), blocks, 8, 2, 1)
        same = all(g.level == r.level and np.array_equal(g.c, r.c) for g, r in zip(got, ref))
        ranks = np.concatenate([ckks.decrypt(P, keys, g)[:8] for g in got])
        err = float(np.max(np.abs(ranks - C.brute_fractional_rank(v))))
        out.put((rank, same, err, len(blocked_dist.pair_partition(3, world)[rank])))
    finally:
        dist.destroy_process_group()


def test_pair_partition_covers_every_pair_once():
    for L in (1, 2, 3, 5, 8):
        for world in (1, 2, 3, 4):
            parts = blocked_dist.pair_partition(L, world)
            flat = [p for part in parts for p in part]
            assert sorted(flat) == [(i, j) for i in range(L) for j in range(i, L)]
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.slow
def test_two_ranks_blocked_rank_equals_single_process():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (same, err, n)) for r, same, err, n in (q.get(timeout=600) for _ in procs))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in (0, 1):
        same, err, n = res[r]
        assert same, f"rank {r}: distributed blocked rank differs from the single-process one"
        assert err < 0.5
        assert n == 3            # 6 block pairs, 3 a rank
