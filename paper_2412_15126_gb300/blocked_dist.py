"""Blocked ranking over several processes, one GPU each (Alg. 7 across devices).

Sec. 5 evaluates the L(L+1)/2 block comparisons C_{i,j} (j >= i) of a vector split into
L blocks as a parallel loop.  Across devices each rank evaluates a share of the block
pairs and the per-block partial sums (rk_rank_blocked_partial), the ranks exchange
their 2L partial-sum ciphertexts once (an all-gather of the canonical coefficient
form through torch.distributed), every rank adds the parts up and assembles the ranks
(rk_rank_blocked_finish).  Additions of residues are exact, so the result is
bit-identical to rk_rank_blocked on one device, whatever the partition.

The functions take an evaluator with five methods, so that the partition and the
exchange do not depend on where the ciphertexts live: `partial(blocks, pairs)`,
`finish(A, B)`, `add(a, b)`, `export(ct)` (a uint64 array [2][level+1][n]) and
`import_(array, like)`.  `CudaEvaluator` is the one over this library's C ABI.
"""
from __future__ import annotations

import numpy as np


def pair_partition(L: int, world: int):
    """The block pairs (i, j), i <= j < L, dealt round-robin to `world` ranks: every
    pair exactly once, shares within one pair of each other."""
    pairs = [(i, j) for i in range(L) for j in range(i, L)]
    return [pairs[r::world] for r in range(world)]


class CudaEvaluator:
    """The evaluator of one rankfhe.Context for blocks of B values (single ciphertexts,
    not stacks; Q packed queries)."""

    def __init__(self, ctx, B: int, Q: int = 1):
        self.ctx = ctx
        self.B = B
        self.Q = Q

    def partial(self, blocks, pairs):
        return self.ctx.rank_blocked_partial(blocks, pairs)

    def finish(self, A, B):
        return self.ctx.rank_blocked_finish(A, B)

    def add(self, a, b):
        return self.ctx.add(a, b)

    def export(self, ct):
        return ct.export()

    def import_(self, arr, like):
        return self.ctx.ct_import(arr, like.level, N=self.B, Q=self.Q, n_real=self.B)


def exchange_sums(ev, parts, rank: int, world: int, group=None):
    """Sum of `parts` (a list of ciphertexts) over every rank: all-gather of the
    exported parts, then each rank adds the others' to its own in rank order."""
    if world == 1:
        return parts
    import torch
    import torch.distributed as dist
    local = np.stack([ev.export(p) for p in parts])
    t = torch.from_numpy(np.ascontiguousarray(local).view(np.int64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    gathered = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(gathered, t, group=group)
    out = list(parts)
    for r in range(world):
        if r == rank:
            continue
        theirs = gathered[r].cpu().numpy().view(np.uint64).reshape(local.shape)
        out = [ev.add(o, ev.import_(theirs[k], parts[k])) for k, o in enumerate(out)]
    return out


def blocked_rank_distributed(ev, blocks, rank: int, world: int, group=None):
    """Ranks of the blocked vector (fractional ranks of Alg. 7, block i in row 0 of
    blocks[i]) with the block pairs divided between the `world` ranks of the process
    group: each rank evaluates its share, one all-gather of the 2L partial sums, then
    every rank assembles the same L rank blocks."""
    L = len(blocks)
    mine = pair_partition(L, world)[rank]
    A, B = ev.partial(blocks, mine)
    sums = exchange_sums(ev, list(A) + list(B), rank, world, group)
    return ev.finish(sums[:L], sums[L:])
