#!/usr/bin/env python
"""Benchmark of the encrypted 128-element rank (Alg. 3) on one GB300 per process.

Workload: rank of a 128-element vector, values uniform in [0, 1) with pairwise
gap >= 2^-9 (seeded), RNS-CKKS with n = 2^16, 28 limbs (scale 2^45) plus 3
special primes, digits of 3 limbs, comparator g^4 then f^2 (Sec. 2.2).  One step
= one complete rank circuit on one encrypted vector (ReplR, TransR, ReplC, Cmp,
SumR), inputs already resident in HBM; the seeded switching keys (4.4 GB of b
parts) exceed L2, so every step streams them from HBM.

Reported (one JSON line from rank 0):
  value          seconds per rank (CUDA events on the library stream), max over ranks
  e2e            the same through the C-ABI from pinned host ciphertexts, with the
                 host->device import and the device->host export of the result timed
  roofline       the forward NTT's butterflies / its event-timed duration (every
                 fourth timed step's launches), against the issue and the integer-
                 multiplier ceilings; roofline_hbm the same for the key inner product
                 in bytes against the measured HBM copy rate
  cpu_baseline   one complete rank on the oracle (plain CPU RNS-CKKS) on the host cores
  clocks         nvidia-smi SM clocks sampled during the timed region
  gpu_launches   kernels this library launched inside the timed region

`--impl reference` times the oracle itself (the CPU reference of this project) on
the same workload: each step is one complete oracle rank, as many as fit a bounded
host budget (the line reports the steps actually run).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "128-elem encrypted rank latency"
UNIT = "s"
PAPER_RANK128_S = 5.76   # the paper's 128-element rank, 64 threads on a Xeon 8358 (context)
WORKLOAD = dict(log_n=16, n_limbs=28, n_special=3, digit_size=3, log_scale=45, log_q0=60, log_special=61,
                d_g=4, d_f=2, N=128, gap=2.0 ** -9, prime_form=1)


def workload_config(extra=None):
    cfg = {"workload": "rank N=128, n=2^16, 28+3 limbs, scale 2^45, dnum digits of 3, Cmp g^4 f^2",
           "vector_len": WORKLOAD["N"], "ring_degree": 1 << WORKLOAD["log_n"], "limbs": WORKLOAD["n_limbs"],
           "special_primes": WORKLOAD["n_special"], "gap": "2^-9",
           "primes": "k 2^32 + 1" if WORKLOAD.get("prime_form") else "1 mod 2n",
           "l2": "working set larger than L2 (seeded rotation and relinearisation keys, ~4.4 GB of b parts, read every step)"}
    if extra:
        cfg.update(extra)
    return cfg


SMALL_WORKLOAD = dict(log_n=13, n_limbs=14, n_special=1, digit_size=1, log_scale=40, log_q0=40, log_special=61,
                      d_g=2, d_f=1, N=8, gap=0.05)


def small_rank_workload(stream, device, reps=20):
    """Rank of an 8-element vector (gap 0.05) at n = 2^13, 14 limbs + 1 special prime,
    Cmp g^2 f^1: latency with inputs resident, CUDA events on the library stream."""
    import numpy as np
    import torch
    from paper_2412_15126_gb300 import inputs, rankfhe
    from oracle.circuits import brute_fractional_rank
    W = SMALL_WORKLOAD
    ctx = rankfhe.Context(W["log_n"], W["n_limbs"], W["n_special"], W["digit_size"], W["log_scale"], W["log_q0"],
                          W["log_special"], W["d_g"], W["d_f"], device=device, stream=stream.cuda_stream,
                          prime_form=W.get("prime_form", 0))
    try:
        ctx.keygen(808, W["N"])
        vecs = [inputs.gap_vector(W["N"], W["gap"], 900 + i) for i in range(reps + 3)]
        cts = [ctx.encrypt(v, N=W["N"]) for v in vecs]
        for ct in cts[:3]:
            ctx.rank(ct).free()
        ctx.sync()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            outs = [ctx.rank(ct) for ct in cts[3:]]
            ev1.record(stream)
        ev1.synchronize()
        err = max(float(np.max(np.abs(ctx.decrypt(o) - brute_fractional_rank(v)))) for o, v in zip(outs, vecs[3:]))
        return {"workload": "rank N=8, gap 0.05, n=2^13, 14 limbs + 1 special, scale 2^40, Cmp g^2 f^1",
                "ms": ev0.elapsed_time(ev1) / reps, "max_rank_error": err}
    finally:
        ctx.close()


def cheb_comparator_workload(stream, device, depths=(8, 10, 12), reps=3):
    """Rank of 128 uniform values with the Chebyshev-approximated comparison (Sec. 2.2)
    at several comparison depths (App. B, Fig. 6): latency with inputs resident (CUDA
    events on the library stream) and the mean / max rank error, n = 2^16, 28 limbs."""
    import numpy as np
    import torch
    from paper_2412_15126_gb300 import rankfhe
    from oracle.circuits import brute_fractional_rank
    W = WORKLOAD
    out = {"workload": "rank N=128, uniform values in [0, 1), n=2^16, 28+3 limbs, scale 2^45, Chebyshev comparator"}
    rng = np.random.default_rng(606)
    vecs = [rng.uniform(0, 1, W["N"]) for _ in range(reps + 1)]
    for d in depths:
        ctx = rankfhe.Context(W["log_n"], W["n_limbs"], W["n_special"], W["digit_size"], W["log_scale"], W["log_q0"],
                              W["log_special"], 0, 0, device=device, stream=stream.cuda_stream, cmp_cheb=1 << (d - 1),
                              prime_form=W.get("prime_form", 0))
        try:
            ctx.keygen(700 + d, W["N"])
            cts = [ctx.encrypt(v, N=W["N"]) for v in vecs]
            ctx.rank(cts[0]).free()
            ctx.sync()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                ev0.record(stream)
                outs = [ctx.rank(ct) for ct in cts[1:]]
                ev1.record(stream)
            ev1.synchronize()
            errs = np.concatenate([np.abs(ctx.decrypt(o) - brute_fractional_rank(v)) for o, v in zip(outs, vecs[1:])])
            out[f"depth{d}"] = {"coefficients": 1 << (d - 1), "ms": ev0.elapsed_time(ev1) / reps,
                                "mean_rank_error": float(errs.mean()), "max_rank_error": float(errs.max())}
        finally:
            ctx.close()
    return out


ORDER_WORKLOAD = dict(log_n=16, n_limbs=34, n_special=3, digit_size=3, log_scale=45, log_q0=60, log_special=61,
                      d_g=3, d_f=2, N=128, levels=64, prime_form=1)


def order_sort_workload(stream, device, reps=3, seed=3):
    """Tie-corrected argmin (Alg. 4, one-hot at the first minimum), argmax with every
    tied maximum (Cmp_G route) and the column-form sort (Alg. 5) of N = 128 values
    on a 64-level grid, n = 2^16 with 34 limbs; inputs resident, each op timed with
    CUDA events on the library stream over `reps` fresh inputs."""
    import numpy as np
    import torch
    from paper_2412_15126_gb300 import inputs, rankfhe

    W = ORDER_WORKLOAD
    ctx = rankfhe.Context(W["log_n"], W["n_limbs"], W["n_special"], W["digit_size"], W["log_scale"], W["log_q0"],
                          W["log_special"], W["d_g"], W["d_f"], device=device, stream=stream.cuda_stream,
                          prime_form=W.get("prime_form", 0))
    try:
        ctx.keygen(5000 + seed, W["N"])
        vecs = [inputs.grid_vector(W["N"], W["levels"], 100 + seed * 10 + i) for i in range(reps + 1)]
        cts = [ctx.encrypt(v, N=W["N"]) for v in vecs]
        ops = {
            "argmin_first": lambda ct: ctx.order_stat(ct, 1, rankfhe.TIES_FIRST),
            "argmax_all": lambda ct: ctx.order_stat(ct, W["N"], rankfhe.TIES_ALL),
            "sort": lambda ct: ctx.sort(ct),
            "median": lambda ct: ctx.median(ct),
        }
        exact = {
            "argmin_first": lambda v: np.eye(len(v))[int(np.argmin(v))],
            "argmax_all": lambda v: (v == v.max()).astype(float),
            "sort": lambda v: np.sort(v),
            "median": lambda v: np.median(v),
        }
        out = {"workload": "N=128 on a 64-level grid (ties), n=2^16, 34+3 limbs, scale 2^45, Cmp g^3 f^2, "
                           "indicator degree 1023"}
        for name, fn in ops.items():
            fn(cts[0]).free()          # warm-up: masks, indicator coefficients
            ctx.sync()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            res = []
            with torch.cuda.stream(stream):
                ev0.record(stream)
                for ct in cts[1:]:
                    res.append(fn(ct))
                ev1.record(stream)
            ev1.synchronize()
            if name == "median":   # the value sits in slot 0
                err = max(abs(float(ctx.decrypt(r)[0]) - exact[name](v)) for r, v in zip(res, vecs[1:]))
            else:
                err = max(float(np.max(np.abs(ctx.decrypt(r) - exact[name](v)))) for r, v in zip(res, vecs[1:]))
            out[name] = {"ms": ev0.elapsed_time(ev1) / reps, "max_error": err}
            for r in res:
                r.free()
        return out
    finally:
        ctx.close()


def blocked_packing_workload(stream, device, reps=1):
    """Blocked rank, argmin and sort of 512 values (4 blocks of 128, Alg. 7, Alg. 4 on
    blocked ranks, Alg. 8) at n = 2^16, 39 + 3 limbs, scale 2^40, Cmp g^4 f^2, values
    distinct with gap >= 2^-9: latency with the block-pair work packed two to a
    ciphertext (RK_OPT_PAIR_PACKING, the rotation by n/4 keyed) and without; CUDA events
    on the library stream, inputs resident."""
    import numpy as np
    import torch
    from paper_2412_15126_gb300 import inputs, rankfhe
    from oracle.circuits import brute_fractional_rank, brute_tie_corrected_rank   # brute-force definitions only
    W = SERVE_SORT
    ctx = rankfhe.Context(W["log_n"], W["n_limbs"], W["n_special"], W["digit_size"], W["log_scale"], W["log_q0"],
                          W["log_special"], W["d_g"], W["d_f"], device=device, stream=stream.cuda_stream,
                          prime_form=W.get("prime_form", 0))
    try:
        ctx.keygen(4321, 128)
        ctx.keygen_rotations([ctx.n // 4])
        v = inputs.gap_vector(512, 2.0 ** -9, 4322)
        blocks = [ctx.encrypt(v[128 * b:128 * (b + 1)], N=128) for b in range(4)]
        ops = {
            "rank": (lambda: ctx.rank_blocked(blocks), brute_fractional_rank(v)),
            "argmin": (lambda: ctx.order_stat_blocked(blocks, 1), np.eye(512)[int(np.argmin(v))]),
            "sort": (lambda: ctx.sort_blocked(blocks), np.sort(v)),
        }
        out = {"workload": "N=512 as 4 blocks of 128, gap 2^-9, n=2^16, 39+3 limbs, scale 2^40, Cmp g^4 f^2, "
                           "indicator 4096 coefficients"}
        for name, (fn, want) in ops.items():
            res = {}
            for packed in (1, 0):
                ctx.set_option(rankfhe.OPT_PAIR_PACKING, packed)
                for r in fn():
                    r.free()            # warm-up: masks, scratch
                ctx.sync()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    e0.record(stream)
                    for _ in range(reps):
                        got = fn()
                    e1.record(stream)
                e1.synchronize()
                dec = np.concatenate([ctx.decrypt(g) for g in got])
                res["packed" if packed else "unpacked"] = {"ms": e0.elapsed_time(e1) / reps,
                                                           "max_error": float(np.max(np.abs(dec - want)))}
            res["speedup"] = res["unpacked"]["ms"] / res["packed"]["ms"]
            out[name] = res
        ctx.set_option(rankfhe.OPT_PAIR_PACKING, 1)
        return out
    finally:
        ctx.close()


RING17 = dict(log_n=17, n_limbs=44, n_special=3, digit_size=3, log_scale=50, log_q0=60, log_special=61, d_g=5, d_f=2,
              prime_form=1)


def blocked_scaling_workload(stream, device, sizes=(512, 2048, 8192, 16384), n17=2048):
    """Blocked ranks (Alg. 7) of N = 512 .. 16384 uniform values on the 128-element
    rank's parameter set (n = 2^16, 28 + 3 limbs, blocks of 128, two block pairs a
    ciphertext), and the blocked argmin and sort (Alg. 4 on the blocked tie-corrected
    ranks, Alg. 8) of N = 2048 values on a 2048-level grid on an n = 2^17 ring (44 + 3
    limbs at 2^50, comparator g^5 f^2, blocks of 128, four block pairs a ciphertext,
    indicator of 16384 coefficients): one run each, CUDA events on the library stream,
    inputs resident; errors against brute force (mean and max for the ranks of
    uniform values, where pairs closer than the comparator resolves swap: the noiseless
    slot model gives the same errors).  The n = 2^17 ring takes the scale 2^50: its
    16384-coefficient indicator squares its Chebyshev terms 13 times, which multiplies
    the rescaling noise by about 4^13, too much at 2^40."""
    import numpy as np
    import torch
    from paper_2412_15126_gb300 import inputs, rankfhe
    from oracle.circuits import brute_fractional_rank   # brute-force definition only

    def run(fn):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            out = fn()
            ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1), out

    out = {"workload": "blocked rank of N uniform values at n=2^16 28+3 limbs (blocks of 128); blocked argmin "
                       "and sort of %d grid values at n=2^17 44+3 limbs 2^50, Cmp g^5 f^2" % n17}
    W = WORKLOAD
    ctx = rankfhe.Context(W["log_n"], W["n_limbs"], W["n_special"], W["digit_size"], W["log_scale"], W["log_q0"],
                          W["log_special"], W["d_g"], W["d_f"], device=device, stream=stream.cuda_stream,
                          prime_form=W.get("prime_form", 0))
    try:
        ctx.keygen(7001, 128)
        ctx.keygen_rotations([ctx.n // 4])       # two block pairs a ciphertext
        rng = np.random.default_rng(7002)
        ranks = {}
        for N in sizes:
            v = rng.uniform(0, 1, N)
            blocks = [ctx.encrypt(v[128 * b:128 * (b + 1)], N=128) for b in range(N // 128)]
            ctx.sync()
            ms, res = run(lambda: ctx.rank_blocked(blocks))
            err = np.abs(np.concatenate([ctx.decrypt(r) for r in res]) - brute_fractional_rank(v))
            ranks[str(N)] = {"s": ms / 1000.0, "mean_rank_error": float(err.mean()), "max_rank_error": float(err.max())}
            for x in res + blocks:
                x.free()
        out["rank_n2^16"] = ranks
    finally:
        ctx.close()
    W = RING17
    ctx = rankfhe.Context(W["log_n"], W["n_limbs"], W["n_special"], W["digit_size"], W["log_scale"], W["log_q0"],
                          W["log_special"], W["d_g"], W["d_f"], device=device, stream=stream.cuda_stream,
                          prime_form=W.get("prime_form", 0))
    try:
        ctx.keygen(7003, 128)
        ctx.keygen_rotations([16384, 32768])     # four block pairs a ciphertext
        v = inputs.grid_vector(n17, n17, 7004)
        blocks = [ctx.encrypt(v[128 * b:128 * (b + 1)], N=128) for b in range(n17 // 128)]
        ctx.sync()
        ms, res = run(lambda: ctx.order_stat_blocked(blocks, 1))
        first = np.zeros(n17)
        first[int(np.argmin(v))] = 1
        e_min = float(np.max(np.abs(np.concatenate([ctx.decrypt(r) for r in res]) - first)))
        ms2, res2 = run(lambda: ctx.sort_blocked(blocks))
        e_sort = float(np.max(np.abs(np.concatenate([ctx.decrypt(r) for r in res2]) - np.sort(v))))
        out["n2^17_%d" % n17] = {"argmin_s": ms / 1000.0, "argmin_max_error": e_min,
                                 "sort_s": ms2 / 1000.0, "sort_max_error": e_sort}
    finally:
        ctx.close()
    return out


def large_argmin(N: int, levels: int = 2048):
    """The blocked argmin (Alg. 4 on the blocked tie-corrected ranks, Alg. 7) of N
    values on a `levels`-level grid (ties) on the n = 2^17 ring (44 + 3 limbs at 2^50,
    comparator g^5 f^2, blocks of 128, four block pairs a ciphertext, indicator of
    8N coefficients): one run, CUDA events on the library stream, inputs resident;
    the one-hot mask against brute force.  Not part of the default run (minutes at
    N = 16384); prints one JSON line."""
    import numpy as np
    import torch
    from paper_2412_15126_gb300 import inputs, rankfhe
    W = RING17
    stream = torch.cuda.Stream()
    ctx = rankfhe.Context(W["log_n"], W["n_limbs"], W["n_special"], W["digit_size"], W["log_scale"], W["log_q0"],
                          W["log_special"], W["d_g"], W["d_f"], device=0, stream=stream.cuda_stream,
                          prime_form=W.get("prime_form", 0))
    try:
        ctx.keygen(7003, 128)
        ctx.keygen_rotations([16384, 32768])     # four block pairs a ciphertext
        v = inputs.grid_vector(N, levels, 7005)
        blocks = [ctx.encrypt(v[128 * b:128 * (b + 1)], N=128) for b in range(N // 128)]
        t0 = time.perf_counter()
        ncoef = len(ctx.indicator_export(N))     # the host computes and caches them: not timed
        coef_s = time.perf_counter() - t0
        ctx.sync()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            res = ctx.order_stat_blocked(blocks, 1)
            ev1.record(stream)
        ev1.synchronize()
        first = np.zeros(N)
        first[int(np.argmin(v))] = 1
        got = np.concatenate([ctx.decrypt(r) for r in res])
        out = {"large_argmin": {"N": N, "grid_levels": levels, "blocks": N // 128, "s": ev0.elapsed_time(ev1) / 1000.0,
                                "indicator_coefficients": ncoef, "indicator_host_s": coef_s,
                                "max_error": float(np.max(np.abs(got - first))),
                                "argmax_of_mask_is_first_minimum": int(np.argmax(got)) == int(np.argmin(v)),
                                "workload": "n=2^17 44+3 limbs 2^50, primes k 2^32 + 1, Cmp g^5 f^2, blocks of 128"}}
        print(json.dumps(out))
    finally:
        ctx.close()
    return 0


# ---------------------------------------------------------------------------
# serving: Poisson arrivals of mixed rank / argmin / sort requests
# ---------------------------------------------------------------------------
SERVE_RANK = dict(log_n=16, n_limbs=34, n_special=3, digit_size=3, log_scale=45, log_q0=60, log_special=61, d_g=4, d_f=2,
                  prime_form=1)
SERVE_SORT = dict(log_n=16, n_limbs=39, n_special=3, digit_size=3, log_scale=40, log_q0=60, log_special=61, d_g=4, d_f=2)
SERVE_LANES = 2   # execution lanes of each serving loop


def serving_requests(count, rate, seed=5, sort_cap=512):
    """Seeded request stream: exponential inter-arrival gaps (mean 1/rate), the op
    uniform over {rank, argmin, sort}, N = round(exp(U(ln 8, ln 1024))) padded to
    2^k (blocks of 128 above 128), values on a 256-level grid.  Sorts are capped at
    sort_cap elements (deeper ones do not fit the 128-bit-secure ring)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        op = ("rank", "argmin", "sort")[int(rng.integers(0, 3))]
        N = int(round(float(np.exp(rng.uniform(np.log(8), np.log(1024))))))
        if op == "sort":
            N = min(N, sort_cap)
        Np = 1 << max(3, (N - 1).bit_length())
        v = rng.integers(0, 256, N) / 256.0
        out.append({"t": t, "op": op, "N": N, "Np": Np, "v": v})
    return out


def serving_workload(stream_a, stream_b, device, count=120, rate=20.0):
    """Two contexts, each with its serving loop (SERVE_LANES execution lanes, continuous
    batching, slot packing of short requests):
    34 limbs at 2^45 for ranks and argmins up to 128 elements, 39 limbs at 2^40 for
    sorts and blocked argmins.  Inputs are
    encrypted before the clock starts; a client thread submits each request at its
    arrival time.  Latency is submit to result on the device (server side)."""
    import threading
    import numpy as np
    from paper_2412_15126_gb300 import rankfhe
    from oracle.circuits import brute_fractional_rank   # brute-force definitions only

    def make(P, stream):
        return rankfhe.Context(P["log_n"], P["n_limbs"], P["n_special"], P["digit_size"], P["log_scale"], P["log_q0"],
                               P["log_special"], P["d_g"], P["d_f"], device=device, stream=stream.cuda_stream,
                               prime_form=P.get("prime_form", 0))

    reqs = serving_requests(count, rate)
    ca, cs = make(SERVE_RANK, stream_a), make(SERVE_SORT, stream_b)
    try:
        ca.keygen(501, 128)
        cs.keygen(502, 128)
        # client encoding: values v -> v/2 in [0, 1/2), padding slots 1/2 + min(k, 255)/512,
        # above every value, so padding never changes a real element's rank.  A sort (at most
        # 255 padding slots) gets distinct padding: the tie offset accumulates the comparator's
        # error at a tie once per tied partner, and a cluster of equal padding values would
        # blur the ranks the sort's indicator reads; every gap stays >= 2^-9
        for r in reqs:   # sorts and blocked argmins need the deeper chain
            ctx = cs if (r["op"] == "sort" or (r["op"] == "argmin" and r["Np"] > 128)) else ca
            x = 0.5 + np.minimum(np.arange(r["Np"]) - r["N"], 255).clip(0) / 512.0
            x[:r["N"]] = r["v"] / 2.0
            r["ctx"] = ctx
            if r["Np"] <= 128:
                r["ct"] = ctx.encrypt(x, N=r["Np"])
            else:
                r["ct"] = ctx.stack([ctx.encrypt(x[b * 128:(b + 1) * 128], N=128) for b in range(r["Np"] // 128)])
        for ctx in (ca, cs):
            # slot packing of short requests: rotations by +-N^2 2^k; the circuits' keys
            # cover all of them except +-n/4 (one Galois element)
            ctx.keygen_rotations([ctx.n // 4])
            ctx.set_option(rankfhe.OPT_SERVER_LANES, SERVE_LANES)
            ctx.sync()
            ctx.server_start(24 << 30, 16)
        tickets = [None] * len(reqs)

        def client():
            t0 = time.perf_counter()
            for i, r in enumerate(reqs):
                d = r["t"] - (time.perf_counter() - t0)
                if d > 0:
                    time.sleep(d)
                blocked = r["Np"] > 128
                if r["op"] == "rank":
                    op = rankfhe.OP_RANK_BLOCKED if blocked else rankfhe.OP_RANK
                    tickets[i] = r["ctx"].server_submit(op, r["ct"])
                elif r["op"] == "argmin":
                    op = rankfhe.OP_ORDER_STAT_BLOCKED if blocked else rankfhe.OP_ORDER_STAT
                    tickets[i] = r["ctx"].server_submit(op, r["ct"], arg=1, flags=rankfhe.TIES_FIRST)
                else:
                    op = rankfhe.OP_SORT_BLOCKED if blocked else rankfhe.OP_SORT
                    tickets[i] = r["ctx"].server_submit(op, r["ct"])

        t_start = time.perf_counter()
        th = threading.Thread(target=client)
        th.start()
        th.join()
        outs = [r["ctx"].server_wait(tk) for r, tk in zip(reqs, tickets)]
        wall = time.perf_counter() - t_start
        stats = {"rank_argmin": ca.server_stats(), "sort_deep": cs.server_stats()}
        for k, ctx in (("rank_argmin", ca), ("sort_deep", cs)):
            stats[k].update(ctx.server_stats_lanes())
        lat = sorted(ca.server_latencies() + cs.server_latencies())
        ca.server_stop()
        cs.server_stop()
        # accuracy of every result against the brute-force answer
        err = {"rank": 0.0, "argmin": 0.0, "sort": 0.0}
        bad = []
        for r, o in zip(reqs, outs):
            ctx = r["ctx"]
            if r["Np"] <= 128:
                got = ctx.decrypt(o)
            else:
                got = np.concatenate([ctx.decrypt(part) for part in ctx.unstack(o)])
            got = got[:r["N"]]
            v = r["v"]
            if r["op"] == "sort":
                got = 2.0 * got   # undo the client encoding
            if r["op"] == "rank":
                want = brute_fractional_rank(v)
            elif r["op"] == "argmin":
                want = np.eye(r["N"])[int(np.argmin(v))]
            else:
                want = np.sort(v)
            e = float(np.max(np.abs(got - want)))
            err[r["op"]] = max(err[r["op"]], e)
            if e > 0.25:
                bad.append({"op": r["op"], "N": r["N"], "Np": r["Np"], "error": e})
        # alone and in the mix: requests re-run directly; a stacked (unpacked) result
        # must be bit-identical, a slot-packed one within 1e-3 of the alone decryption
        same, mix_err = True, 0.0
        for r, o in list(zip(reqs, outs))[:6]:
            ctx, blocked = r["ctx"], r["Np"] > 128
            parts = ctx.unstack(r["ct"]) if blocked else None
            if r["op"] == "rank":
                ref = ctx.rank_blocked(parts) if blocked else [ctx.rank(r["ct"])]
            elif r["op"] == "argmin":
                ref = ctx.order_stat_blocked(parts, 1) if blocked else [ctx.order_stat(r["ct"], 1, rankfhe.TIES_FIRST)]
            else:
                ref = ctx.sort_blocked(parts) if blocked else [ctx.sort(r["ct"])]
            got = ctx.unstack(o) if blocked else [o]
            for a, b in zip(got, ref):
                e = float(np.max(np.abs(ctx.decrypt(a)[:r["N"]] - ctx.decrypt(b)[:r["N"]])))
                mix_err = max(mix_err, e)
                if blocked:
                    same = same and np.array_equal(a.export(), b.export())
        sizes = [r["N"] for r in reqs]
        return {
            "requests": len(reqs), "rate_per_s": rate, "wall_s": wall, "requests_per_s": len(reqs) / wall,
            "elements_per_s": sum(sizes) / wall,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)), "max_s": float(lat[-1]),
            "peak_device_bytes_above_start": max(stats["rank_argmin"]["peak_bytes"], stats["sort_deep"]["peak_bytes"]),
            "rank_argmin_server": stats["rank_argmin"], "deep_server": stats["sort_deep"],
            "max_abs_error": err, "requests_over_0.25": bad, "blocked_identical_alone_vs_mix": same,
            "max_decrypted_diff_alone_vs_mix": mix_err, "alone_vs_mix_tolerance": 1e-3,
            "alone_vs_mix_ok": same and mix_err < 1e-3,
            "ops": {op: sum(1 for r in reqs if r["op"] == op) for op in ("rank", "argmin", "sort")},
            "blocked": sum(1 for r in reqs if r["Np"] > 128),
            "workload": "Poisson 20 req/s, op uniform {rank, argmin, sort}, N log-uniform 8..1024 padded to 2^k "
                        "(blocks of 128 above 128, sorts capped at 512), 256-level grid encoded as v/2 with padding "
                        "1/2 + min(k, 255)/512; ranks and argmins <= 128 "
                        "n=2^16 34+3 limbs 2^45, sorts and blocked argmins 39+3 limbs 2^40, Cmp g^4 f^2",
        }
    finally:
        ca.close()
        cs.close()


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for(local_rank: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCE = {   # kernel -> [(file, first line of its source or None, text after it or None)]
    "ks_inner": [("kernels.cu", "// Up to CH stacked ciphertexts per thread", "// out[c][t] = base_c[t]")],
    "ntt_fwd": [("ntt.cu", None, None), ("ntt_core.cuh", None, None)],
}


def kernel_source_sha256(kernel: str):
    h = hashlib.sha256()
    for f, a, b in KERNEL_SOURCE[kernel]:
        src = open(os.path.join(ROOT, "paper_2412_15126_gb300", "csrc", f)).read()
        if a is not None:
            i = src.index(a)
            src = src[i:src.index(b, i)].rstrip()
        h.update(src.encode())
    return h.hexdigest()


GB300_SMS, GB300_SCHEDULERS, GB300_MAX_SM_MHZ = 152, 4, 2070.0


PROF_EVERY = 4   # timed steps whose kernel launches the roofline events bracket: every 4th


def ntt_roofline(prof, clk, alu=None):
    """Forward NTT (both passes), the dominant kernel: bound by integer arithmetic, so
    the ceiling is the device's measured butterfly rate (rk_measure_alu: the same
    Cooley-Tukey butterfly with its operands in registers, no memory traffic, over
    every SM).  achieved = butterflies per launch / CUDA-event launch duration.  Also
    reported: the SMs' issue rate (152 SMs x 4 schedulers x one warp instruction a
    clock at the maximum SM clock) divided by the instructions one butterfly costs in
    this kernel (ncu capture in profiles/traffic.json), and the integer-multiplier
    pipe's rate over its busy cycles a butterfly."""
    if not prof["launches"] or prof["ms"] <= 0:
        return None
    per_launch = prof["ops"] / prof["launches"]
    avg_s = prof["ms"] * 1e-3 / prof["launches"]
    achieved = per_launch / avg_s / 1e9
    ipb = hpb = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)["ntt_fwd"]
        if rec["source_sha256"] == kernel_source_sha256("ntt_fwd"):   # counts of this very kernel
            ipb = rec["thread_instructions_per_butterfly"]
            hpb = rec.get("fmaheavy_cycles_per_butterfly")
    except Exception:
        pass
    peak = mul_peak = None
    if ipb:
        peak = GB300_SMS * GB300_SCHEDULERS * 32 * GB300_MAX_SM_MHZ * 1e6 / ipb / 1e9
    if hpb:
        # the integer multiplier (FMA-heavy) pipe: one busy cycle of each of the 608
        # sub-partitions per clock, hpb busy cycles a butterfly
        mul_peak = GB300_SMS * GB300_SCHEDULERS * GB300_MAX_SM_MHZ * 1e6 / hpb / 1e9
    # the transforms run the general butterfly for every prime form
    bpeak = alu["butterfly_per_s"] / 1e9 if alu and alu.get("butterfly_per_s") else None
    return {"bound": "alu", "kernel": "ntt_fwd (column + row pass)", "achieved": achieved, "peak": bpeak,
            "peak_kind": "measured: register-resident Cooley-Tukey butterflies a second over every SM "
                         "(rk_measure_alu microbenchmark)", "unit": "Gbutterfly/s",
            "frac": (achieved / bpeak) if bpeak else None,
            "issue_peak": peak, "issue_frac": (achieved / peak) if peak else None,
            "issue_peak_kind": "derived: 152 SMs x 4 schedulers x 1 warp instruction/clock x 2070 MHz / "
                               "instructions per butterfly of this kernel (ncu)",
            "multiplier_pipe_peak": mul_peak, "multiplier_pipe_frac": (achieved / mul_peak) if mul_peak else None,
            "traffic": committed_traffic("ntt_fwd", prof["bytes"] / prof["launches"]),
            "algorithmic_bytes_per_launch": prof["bytes"] / prof["launches"], "butterflies_per_launch": per_launch,
            "avg_launch_us": avg_s * 1e6, "launches": prof["launches"],
            "sm_mhz_under_load": (clk or {}).get("sm_mhz")}


def ks_algorithmic(limbs: int, log_n: int = 16, alpha: int = 3, dsize: int = 3, seeded: bool = True):
    """Algorithmic cost of one hybrid key switch at `limbs` = l+1 live limbs: bytes =
    8n [2(l+1) input + parts beta (l+1+alpha) key + 2(l+1) output], parts = 1 for seeded
    keys (the a parts regenerated, so the key stream is the b parts), 2 for explicit
    keys; modular products = (n/2) log2 n [beta (l+1+alpha) + 2(l+1) + 2 alpha]
    butterflies of the transforms plus n [3 beta (l+1) + 6(l+1) + 2 beta (l+1+alpha)] of
    the conversions and the inner product."""
    n = 1 << log_n
    beta = -(-limbs // dsize)
    qp = limbs + alpha
    bytes_ = 8 * n * (2 * limbs + (1 if seeded else 2) * beta * qp + 2 * limbs)
    modmuls = (n // 2) * log_n * (beta * qp + 2 * limbs + 2 * alpha) + n * (3 * beta * limbs + 6 * limbs + 2 * beta * qp)
    return bytes_, modmuls


def keyswitch_roofline(ctx, stream, alu, hbm_peak, reps=10):
    """One complete key switch (a rotation: ModUp with its transforms, the key inner
    product, ModDown with its transforms and the combine) at 28, 18 and 9 limbs,
    timed with CUDA events on the library stream around `reps` back-to-back
    rotations of a resident ciphertext: algorithmic bytes and modular products per
    switch over its average duration, against the measured HBM copy rate and the
    measured modular-product rate."""
    import torch
    from paper_2412_15126_gb300 import inputs
    W = WORKLOAD
    ct = ctx.encrypt(inputs.gap_vector(W["N"], W["gap"], 77), N=W["N"])
    out = {}
    for limbs in (28, 18, 9):
        x = ct
        while x.level + 1 > limbs:
            x = ctx.mul_scalar(x, 1.0)
        for _ in range(2):
            ctx.rotate(x, -W["N"]).free()
        ctx.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        res = []
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                res.append(ctx.rotate(x, -W["N"]))
            e1.record(stream)
        e1.synchronize()
        us = e0.elapsed_time(e1) * 1000.0 / reps
        for r in res:
            r.free()
        b, m = ks_algorithmic(limbs)
        gbs = b / (us * 1e-6) / 1e9
        gmm = m / (us * 1e-6) / 1e9
        out[str(limbs)] = {"us": us, "algorithmic_mb": b / 1e6, "gb_per_s": gbs, "frac_hbm": gbs / hbm_peak,
                           "gmodmul_per_s": gmm,
                           "frac_modmul_peak": (gmm * 1e9 / alu["modmul_per_s"]) if alu else None}
    return out


def committed_traffic(kernel: str, algorithmic_per_launch: float):
    """DRAM bytes per launch from the committed ncu capture (profiles/traffic.json),
    scaled from the captured launch to the timed launches' average by algorithmic
    bytes; None if the kernel's source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)[kernel]
        if d["source_sha256"] != kernel_source_sha256(kernel):
            return None
        return d["dram_bytes"] / d["algorithmic_bytes"] * algorithmic_per_launch
    except Exception:
        return None


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample
# ---------------------------------------------------------------------------
def rank_rotations(N):
    """The rotation amounts of a rank circuit (ReplR, TransR, ReplC, SumR; Sec. 3.1),
    with the sums of the step pairs its chains take two at a time."""
    k = N.bit_length() - 1
    chains = [[-(N << i) for i in range(k)], [-(1 << i) for i in range(k)], [N << i for i in range(k)],
              [-((N * (N - 1)) >> i) for i in range(1, k + 1)]]
    rs = set()
    for ch in chains:   # every step, and the sums of the step pairs taken two at a time
        rs.update(ch)
        rs.update(ch[i] + ch[i + 1] for i in range(0, len(ch) - 1, 2))
    return sorted(rs)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_rank_setup(seed: int = 3):
    """The oracle's parameters, keys (the rank's 28 rotations and relinearisation) and
    one encrypted input of the 128-element workload (none of it timed)."""
    from oracle import ckks
    from paper_2412_15126_gb300 import inputs
    W = WORKLOAD
    P = ckks.gen_params(W["log_n"], W["n_limbs"], W["log_q0"], W["log_scale"], W["n_special"],
                        W["log_special"], W["digit_size"], W.get("prime_form", 0))
    keys = ckks.keygen(P, seed, sorted({ckks.galois_left(r % P.slots, P.n) for r in rank_rotations(W["N"])}))
    v = inputs.gap_vector(W["N"], W["gap"], seed)
    return P, keys, v, ckks.encrypt(P, keys, v, seed)


def oracle_rank_timed(setup, max_ranks: int, budget_s: float):
    """Complete oracle ranks (Alg. 3 on the plain CPU RNS-CKKS, every rotation, product
    and rescale of the circuit) of the 128-element workload, one after another until
    `max_ranks` are done or `budget_s` seconds have passed (at least one).  Returns the
    per-rank seconds and the largest rank error of the decrypted results."""
    import numpy as np
    from oracle import ckks, circuits as C
    P, keys, v, ct = setup
    W = WORKLOAD
    times, err = [], 0.0
    t_all = time.perf_counter()
    while len(times) < max_ranks:
        t0 = time.perf_counter()
        R = C.rank(C.OracleCkks(P, keys), ct, W["N"], W["d_g"], W["d_f"])
        times.append(time.perf_counter() - t0)
        got = ckks.decrypt(P, keys, R)[: W["N"]]
        err = max(err, float(np.max(np.abs(got - C.brute_fractional_rank(v)))))
        if time.perf_counter() - t_all >= budget_s:
            break
    return times, err


def oracle_rank_estimate(steps: int = 1, warmup: int = 0, setup=None):
    """Time the oracle's rotation, product and scalar product at the top level (28
    limbs), `steps` times each, and scale to one full rank circuit: each key switch
    (rotation or product) at level l weighted by beta_l (l+1+alpha) relative to the
    top level, each scalar/mask product by (l+1).  Returns seconds per rank and the
    per-step samples.  A model, kept beside the complete ranks as a cross-check."""
    import numpy as np
    from oracle import ckks, circuits as C

    W = WORKLOAD
    if setup is None:
        P = ckks.gen_params(W["log_n"], W["n_limbs"], W["log_q0"], W["log_scale"], W["n_special"],
                            W["log_special"], W["digit_size"], W.get("prime_form", 0))
        keys = ckks.keygen(P, 3, [ckks.galois_left(P.slots - W["N"], P.n)])
        from paper_2412_15126_gb300 import inputs
        ct = ckks.encrypt(P, keys, inputs.gap_vector(W["N"], W["gap"], 1), 1)
    else:
        P, keys, _, ct = setup

    # op trace of the rank circuit (levels from the noiseless model of the same schedule)
    class Trace(C.PlainSlots):
        def __init__(self, slots, top):
            super().__init__(slots, top)
            self.ops = []

        def rot(self, x, r):
            self.ops.append(("ks", x.level))
            return super().rot(x, r)

        def mul(self, x, y):
            self.ops.append(("ks", x.level))
            return super().mul(x, y)

        def mul_scalar(self, x, c):
            self.ops.append(("rs", x.level))
            return super().mul_scalar(x, c)

        def mul_plain(self, x, key):
            self.ops.append(("rs", x.level))
            return super().mul_plain(x, key)

    T = Trace(P.slots, P.L)
    C.rank(T, T.fresh(np.zeros(W["N"])), W["N"], W["d_g"], W["d_f"])
    top = P.L

    def w_ks(l):
        return P.beta(l) * (l + 1 + P.alpha)

    samples = []
    for s in range(warmup + steps):
        t0 = time.perf_counter()
        ckks.rotate(P, keys, ct, -W["N"])
        t_rot = time.perf_counter() - t0
        t0 = time.perf_counter()
        ckks.mul(P, keys, ct, ct)
        t_mul = time.perf_counter() - t0
        t0 = time.perf_counter()
        ckks.mul_scalar(P, ct, 0.5)
        t_rs = time.perf_counter() - t0
        t_ks = 0.5 * (t_rot + t_mul)
        est = 0.0
        for kind, l in T.ops:
            est += t_ks * w_ks(l) / w_ks(top) if kind == "ks" else t_rs * (l + 1) / (top + 1)
        if s >= warmup:
            samples.append({"est_s": est, "sample_s": t_rot + t_mul + t_rs})
    n_ks = sum(1 for k, _ in T.ops if k == "ks")
    n_rs = len(T.ops) - n_ks
    desc = (f"one rotation, one product (tensor+relinearise+rescale) and one scalar product of a 28-limb "
            f"ciphertext per step on the oracle, scaled to the rank circuit's {n_ks} key switches and {n_rs} "
            f"scalar/mask products by beta_l(l+1+alpha) and (l+1) per level")
    return samples, desc


def cpu_cores():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# batched form: 96 queries of N in {16, 32, 64, 128} + 8 queries of N = 512 (4 blocks)
# ---------------------------------------------------------------------------
def batched_workload(ctx, seed=4):
    """Per-query form (one ciphertext and one circuit per query, blocked queries one
    Alg. 7 each) against the batched form (queries of one length slot-packed Q =
    (n/2)/N^2 per ciphertext, ciphertexts of one shape stacked into one circuit,
    N = 512 queries packed two per block ciphertext).  Inputs resident; both timed
    end of queue to end of queue with CUDA events on the library stream."""
    import numpy as np
    import torch
    from paper_2412_15126_gb300 import inputs
    from oracle.circuits import brute_fractional_rank

    slots = 1 << (WORKLOAD["log_n"] - 1)
    lens = inputs.batch_lengths(96, seed=seed)
    vecs = [inputs.gap_vector(N, WORKLOAD["gap"], 10_000 + i) for i, N in enumerate(lens)]
    big = [inputs.gap_vector(512, WORKLOAD["gap"], 20_000 + i) for i in range(8)]
    pq = [ctx.encrypt(v, N=N) for v, N in zip(vecs, lens)]
    pq_blocks = [[ctx.encrypt(v[128 * b:128 * (b + 1)], N=128) for b in range(4)] for v in big]
    packed, packed_ids, packed_shape = [], [], []
    for N in sorted(set(lens)):
        ids = [i for i, x in enumerate(lens) if x == N]
        qmax = slots // (N * N)
        for s in range(0, len(ids), qmax):
            chunk = ids[s:s + qmax]
            packed.append(ctx.encrypt(np.concatenate([vecs[i] for i in chunk]), N=N, Q=len(chunk), n_real=N))
            packed_ids.append(chunk)
            packed_shape.append((N, len(chunk)))
    pk_blocks = []
    for a in range(0, 8, 2):
        pk_blocks.append([ctx.encrypt(np.concatenate([big[a][128 * b:128 * (b + 1)], big[a + 1][128 * b:128 * (b + 1)]]),
                                      N=128, Q=2, n_real=128) for b in range(4)])
    def timed(fn):
        ctx.sync()
        t0 = time.perf_counter()
        out = fn()
        ctx.sync()
        return time.perf_counter() - t0, out

    # the packed blocked queries as one circuit: block i of every packed pair in one stack
    pk_stacked = [ctx.stack([grp[b] for grp in pk_blocks]) for b in range(4)]
    from paper_2412_15126_gb300 import rankfhe

    def pq_blocked_plain():   # every block and block-pair ciphertext with its own launches
        ctx.set_option(rankfhe.OPT_BLOCK_STACKING, 0)
        try:
            return [ctx.rank_blocked(b) for b in pq_blocks]
        finally:
            ctx.set_option(rankfhe.OPT_BLOCK_STACKING, 1)

    pq_single = lambda: [ctx.rank(c) for c in pq]
    pq_blocked = lambda: [ctx.rank_blocked(b) for b in pq_blocks]
    b_single = lambda: ctx.rank_batch(packed)
    b_blocked = lambda: [[ctx.unstack(o) for o in ctx.rank_blocked(pk_stacked)]]
    for fn in (b_single, b_blocked, pq_single, pq_blocked, pq_blocked_plain):   # warm-up: masks, scratch
        timed(fn)
    t_pqs, _ = timed(pq_single)
    t_pqb, _ = timed(pq_blocked_plain)
    t_pqb_st, _ = timed(pq_blocked)
    t_bs, out_bs = timed(b_single)
    t_bb, out_bb = timed(b_blocked)
    t_pq, t_b = t_pqs + t_pqb, t_bs + t_bb
    out_b = (out_bs, out_bb)
    # the batched form replayed from CUDA graphs: one graph per group of packed
    # ciphertexts of one shape (stacked, as rk_rank_batch groups them) and one for the
    # stack of the packed blocked queries
    groups = {}
    for ct, shape in zip(packed, packed_shape):
        groups.setdefault(shape, []).append(ct)
    g_in = [ctx.stack(g) for g in groups.values()]
    graphs = [ctx.graph_capture(rankfhe.OP_RANK, x) for x in g_in]
    b_in = ctx.stack(pk_stacked)
    gb = ctx.graph_capture(rankfhe.OP_RANK_BLOCKED, b_in, L=4)
    replay = lambda: [g.run(x) for g, x in zip(graphs, g_in)] + [gb.run(b_in)]
    timed(replay)
    t_g, out_g = timed(replay)
    graph_same = bool(np.array_equal(ctx.unstack(out_g[-1])[0].export(), out_bb[0][0][0].export()))
    for g in graphs + [gb]:
        g.free()
    # correctness of the batched outputs
    err = 0.0
    for ct, chunk in zip(out_b[0], packed_ids):
        got = ctx.decrypt(ct).reshape(len(chunk), -1)
        for row, i in zip(got, chunk):
            err = max(err, float(np.max(np.abs(row - brute_fractional_rank(vecs[i])))))
    blocks_by_group = [[out_b[1][0][b][g] for b in range(4)] for g in range(len(pk_blocks))]
    for pair, blocks in zip(range(0, 8, 2), blocks_by_group):
        got = np.stack([ctx.decrypt(b).reshape(2, 128) for b in blocks], axis=1).reshape(2, 512)
        for q in range(2):
            err = max(err, float(np.max(np.abs(got[q] - brute_fractional_rank(big[pair + q])))))
    n_q = len(vecs) + len(big)
    elems = sum(lens) + 512 * len(big)
    return {"queries": n_q, "elements": elems, "per_query_s": t_pq, "batched_s": t_b,
            "per_query_split_s": {"single": t_pqs, "blocked": t_pqb}, "batched_split_s": {"single": t_bs, "blocked": t_bb},
            "per_query_form": "one ciphertext per query, every block and block-pair ciphertext with its own "
                              "launches, no graphs",
            "speedup_vs_per_query_with_stacked_pairs": (t_pqs + t_pqb_st) / t_b,
            "ranks_per_s": n_q / t_b, "per_query_ranks_per_s": n_q / t_pq, "elements_per_s": elems / t_b,
            "speedup": t_pq / t_b, "ciphertexts_batched": len(packed) + 4 * len(pk_blocks),
            "batched_graph_s": t_g, "graph_ranks_per_s": n_q / t_g, "speedup_graph": t_pq / t_g,
            "graphs": len(graphs) + 1, "graph_blocked_bit_identical": graph_same,
            "ciphertexts_per_query": len(pq) + 4 * len(pq_blocks), "max_rank_error": err}


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------
def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest x over all ranks: a replicated job's time is its slowest replica's."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank: int, i: int) -> int:
    """Seed of input i on replica `rank`: every replica ranks its own vectors."""
    return 1 + rank * 1000 + i


REF_BUDGET_S = 120.0   # host seconds the reference arm spends on complete oracle ranks


def run_reference(args):
    """The oracle as it stands on the host cores: complete 128-element ranks, as many
    as --steps asks for or as fit REF_BUDGET_S (at least one); `steps` reports the
    ranks actually timed.  The oracle has nothing to warm up (no caches, no JIT), so
    no untimed ranks run; key generation is outside the timed ranks."""
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    from oracle import _lib
    _lib.build()
    t0 = time.perf_counter()
    setup = oracle_rank_setup()
    keygen_s = time.perf_counter() - t0
    times, err = oracle_rank_timed(setup, args.steps, REF_BUDGET_S)
    value = statistics.mean(times)
    model, desc = oracle_rank_estimate(steps=1, setup=setup)
    sample = (f"{len(times)} complete rank circuit(s) of the 128-element workload on the oracle (28 rotations, "
              f"24 products, every rescale), one encrypted input, keys generated beforehand ({keygen_s:.0f} s, not "
              f"timed); up to --steps ranks within {REF_BUDGET_S:.0f} s")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(times), "warmup": 0, "ms_per_step": value * 1000.0, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": value / PAPER_RANK128_S, "dtype": "u64", "data": "synthetic",
        "config": workload_config({"impl_detail": "plain CPU RNS-CKKS oracle (C core, OpenMP over residues)",
                                   "steps_requested": args.steps, "warmup_requested": args.warmup,
                                   "max_rank_error": err}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": sample,
                         "host_cpu": cpu_model(), "rank_seconds": times,
                         "model_estimate_s": model[0]["est_s"], "model": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_cuda(args):
    import numpy as np
    import torch

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2412_15126_gb300 import inputs, rankfhe

    W = WORKLOAD
    stream = torch.cuda.Stream()
    ctx = rankfhe.Context(W["log_n"], W["n_limbs"], W["n_special"], W["digit_size"], W["log_scale"], W["log_q0"],
                          W["log_special"], W["d_g"], W["d_f"], device=local, stream=stream.cuda_stream,
                          prime_form=W.get("prime_form", 0))
    ctx.keygen(1000 + rank, W["N"])
    tuned = ctx.autotune() if not args.no_autotune else None
    alu = ctx.measure_alu()
    n_in = args.warmup + args.steps
    vecs = [inputs.gap_vector(W["N"], W["gap"], replica_seed(rank, i)) for i in range(n_in)]
    cts = [ctx.encrypt(v, N=W["N"]) for v in vecs]
    ctx.sync()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # warm-up (also builds the cached plaintext masks)
    for i in range(args.warmup):
        ctx.rank(cts[i])
    ctx.sync()
    # the kernel events bracket the launches of every PROF_EVERY-th timed step only
    # (each costs a few microseconds of device time); size the event pool for them
    # here, outside the timed region
    n_prof = (args.steps + PROF_EVERY - 1) // PROF_EVERY
    ctx.profile_start("ntt_fwd,ks_inner")
    for i in range(n_prof):
        ctx.rank(cts[i % max(args.warmup, 1)]).free()
    ctx.profile_stop()

    clocks = ClockSampler(gpu_id_for(local))
    barrier()
    torch.cuda.synchronize()
    ctx.sync()
    clocks.start()
    time.sleep(0.2)
    launches0 = ctx.launch_count()
    ctx.profile_start("ntt_fwd,ks_inner")   # the dominant (issue-bound) and the HBM-bound kernel
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    outs = []
    torch.cuda.nvtx.range_push("timed")
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for i in range(args.steps):
            ctx.profile_pause(i % PROF_EVERY != 0)
            outs.append(ctx.rank(cts[args.warmup + i]))
        ev1.record(stream)
    ev1.synchronize()
    torch.cuda.nvtx.range_pop()
    ctx.sync()
    ctx.profile_stop()
    prof_ntt = ctx.profile_kind("ntt_fwd")
    prof_ks = ctx.profile_kind("ks_inner")
    launches = ctx.launch_count() - launches0
    clk = clocks.stop()
    barrier()
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    ms_per_step = elapsed_ms / args.steps

    # correctness of the timed outputs (outside the timed region)
    from oracle.circuits import brute_fractional_rank  # brute-force definition only
    err = 0.0
    for i in (0, args.steps - 1):
        got = ctx.decrypt(outs[i])
        err = max(err, float(np.max(np.abs(got - brute_fractional_rank(vecs[args.warmup + i])))))
    for o in outs:
        o.free()

    # end to end through the C-ABI: pinned host ciphertexts in, result ciphertext out
    e2e_steps = min(args.steps, 10)
    host_in = []
    for i in range(e2e_steps):
        arr = cts[args.warmup + i].export()
        pinned = torch.empty(arr.size, dtype=torch.int64, pin_memory=True)
        pinned.numpy()[:] = arr.reshape(-1).view(np.int64)
        host_in.append((pinned, arr.shape))
    out_level = None
    barrier()
    ctx.sync()
    t0 = time.perf_counter()
    for pinned, shape in host_in:
        g = ctx.ct_import(pinned.numpy().view(np.uint64).reshape(shape), shape[1] - 1, N=W["N"])
        r = ctx.rank(g)
        res = r.export()                      # device -> host read of the result
        out_level = r.level
        g.free()
        r.free()
    ctx.sync()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
    n = 1 << W["log_n"]
    h2d = 2 * W["n_limbs"] * n * 8
    d2h = 2 * (out_level + 1) * n * 8 if out_level is not None else 0

    # per kernel kind: algorithmic bytes over event-timed duration, one profiled rank step
    kinds = None
    if not args.no_kernel_table:
        kinds = {}
        names = ("ntt_fwd", "ntt_inv", "modup", "ks_inner", "moddown_conv", "ks_combine", "tensor", "rescale",
                 "pointwise")
        ctx.sync()
        ctx.profile_start(",".join(names))
        ctx.rank(cts[args.warmup]).free()
        ctx.profile_stop()
        for kind in names:
            pr = ctx.profile_kind(kind)
            if pr["launches"]:
                gbs = pr["bytes"] / (pr["ms"] * 1e-3) / 1e9
                kinds[kind] = {"launches": pr["launches"], "ms_per_step": pr["ms"], "gb": pr["bytes"] / 1e9,
                               "gbs": gbs, "frac_hbm": gbs / measured_peaks()[0]}

    # the same steps replayed from one CUDA graph of the rank circuit
    graph = None
    if not args.no_graph:
        g = ctx.graph_rank(cts[0])
        for i in range(args.warmup):
            g.run(cts[i]).free()
        ctx.sync()
        gev0 = torch.cuda.Event(enable_timing=True)
        gev1 = torch.cuda.Event(enable_timing=True)
        gouts = []
        with torch.cuda.stream(stream):
            gev0.record(stream)
            for i in range(args.steps):
                gouts.append(g.run(cts[args.warmup + i]))
            gev1.record(stream)
        gev1.synchronize()
        same = bool(np.array_equal(gouts[-1].export(), ctx.rank(cts[args.warmup + args.steps - 1]).export()))
        graph = {"ms_per_step": gev0.elapsed_time(gev1) / args.steps, "bit_identical_to_direct": same}
        for o in gouts:
            o.free()
        g.free()

    # the same rank with the input first brought down to the lowest level the circuit
    # needs (RK_OPT_TRIM_LEVELS): the same work on fewer limbs, result at level 0
    trimmed = None
    if not args.no_graph:
        ctx.set_option(rankfhe.OPT_TRIM_LEVELS, 1)
        try:
            for i in range(args.warmup):
                ctx.rank(cts[i]).free()
            ctx.sync()
            tev0 = torch.cuda.Event(enable_timing=True)
            tev1 = torch.cuda.Event(enable_timing=True)
            touts = []
            with torch.cuda.stream(stream):
                tev0.record(stream)
                for i in range(args.steps):
                    touts.append(ctx.rank(cts[args.warmup + i]))
                tev1.record(stream)
            tev1.synchronize()
            terr = max(float(np.max(np.abs(ctx.decrypt(touts[i]) - brute_fractional_rank(vecs[args.warmup + i]))))
                       for i in (0, args.steps - 1))
            trimmed = {"ms_per_step": tev0.elapsed_time(tev1) / args.steps, "out_level": touts[0].level,
                       "max_rank_error": terr,
                       "note": "opt-in: input brought down to the level the circuit needs before the rank"}
            for o in touts:
                o.free()
        finally:
            ctx.set_option(rankfhe.OPT_TRIM_LEVELS, 0)

    batched = None
    if not args.no_batched:
        batched = batched_workload(ctx)

    order_sort = None
    small = None
    cheb = None
    if not args.no_order_sort and world == 1:
        order_sort = order_sort_workload(stream, local)
        small = small_rank_workload(stream, local)
        cheb = cheb_comparator_workload(stream, local)

    blocked = scaling = None
    if not args.no_order_sort and world == 1:
        blocked = blocked_packing_workload(stream, local)
        scaling = blocked_scaling_workload(stream, local)

    serving = None
    if args.serve and world == 1:
        serving = serving_workload(stream, torch.cuda.Stream(), local, count=args.serve)

    peak, peak_kind = measured_peaks()
    keyswitch = None
    if not args.no_kernel_table:
        keyswitch = keyswitch_roofline(ctx, stream, alu, peak)
    roof_ntt = ntt_roofline(prof_ntt, clk, alu)
    sampled = "launches of every %dth timed step (%d of %d steps)" % (PROF_EVERY, n_prof, args.steps)
    if roof_ntt:
        roof_ntt["events_on"] = sampled
    ks_achieved = prof_ks["bytes"] / (prof_ks["ms"] * 1e-3) / 1e9 if prof_ks["launches"] and prof_ks["ms"] > 0 else None
    roof_ks = {"bound": "hbm", "kernel": "ks_inner", "achieved": ks_achieved, "peak": peak, "peak_kind": peak_kind,
               "unit": "GB/s", "frac": (ks_achieved / peak) if ks_achieved else None,
               "traffic": committed_traffic("ks_inner", prof_ks["bytes"] / max(prof_ks["launches"], 1)),
               "algorithmic_bytes_per_launch": prof_ks["bytes"] / max(prof_ks["launches"], 1),
               "avg_launch_us": prof_ks["ms"] * 1000.0 / max(prof_ks["launches"], 1), "launches": prof_ks["launches"],
               "events_on": sampled}

    line = None
    if rank == 0:
        value = ms_per_step / 1000.0
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            setup = oracle_rank_setup()
            times, cerr = oracle_rank_timed(setup, 1, 0.0)
            cpu = {"value": times[0], "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                   "sample": "one complete rank circuit of the 128-element workload on the oracle (28 rotations, 24 "
                             "products, every rescale), keys generated beforehand (not timed)",
                   "host_cpu": cpu_model(), "max_rank_error": cerr}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": value / PAPER_RANK128_S, "dtype": "u64", "data": "synthetic",
            "config": workload_config({"ranks_per_s_total": world * 1000.0 / ms_per_step,
                                       "max_rank_error": err}),
            "e2e": {"value": e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": roof_ntt,
            "roofline_hbm": roof_ks,
            "keyswitch": keyswitch,
            "alu_peaks": alu,
            "cpu_baseline": cpu,
            "batched": batched,
            "graph": graph, "trimmed_levels": trimmed,
            "order_sort": order_sort,
            "blocked_512": blocked,
            "blocked_scaling": scaling,
            "rank8": small,
            "cheb_comparator": cheb,
            "serving": serving,
            "autotune": tuned,
            "kernels": kinds,
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    for c in cts:
        c.free()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def profile_case(ntt_group_mib=0, modup_col=False):
    """Small case for ncu captures: the rank workload's parameters (n = 2^16, 28 + 3
    limbs) but only the keys of one rotation (about 1.3 GB on the device); two top-level
    rotations and one product inside the NVTX range "prof".  ntt_group_mib and
    modup_col set the launch options the autotuner chose in the timed run."""
    import numpy as np
    import torch
    from paper_2412_15126_gb300 import rankfhe
    W = WORKLOAD
    ctx = rankfhe.Context(W["log_n"], W["n_limbs"], W["n_special"], W["digit_size"], W["log_scale"], W["log_q0"],
                          W["log_special"], W["d_g"], W["d_f"], device=0, prime_form=W.get("prime_form", 0))
    ctx.set_option(rankfhe.OPT_NTT_GROUP_BYTES, ntt_group_mib << 20)
    ctx.set_option(rankfhe.OPT_MODUP_COL, 1 if modup_col else 0)
    ctx.keygen(5, 2)
    ct = ctx.encrypt(np.linspace(0.0, 0.9, 2), N=2)
    ctx.sync()
    torch.cuda.nvtx.range_push("prof")
    for _ in range(2):
        r = ctx.rotate(ct, -2)
    m = ctx.mul(ct, ct)
    ctx.sync()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_case": "ok", "levels": [r.level, m.level]}))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 104-query batched workload")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay of the rank steps")
    ap.add_argument("--no-kernel-table", action="store_true", help="skip the per-kernel-kind roofline table")
    ap.add_argument("--no-order-sort", action="store_true", help="skip the 34-limb argmin/argmax/sort latencies")
    ap.add_argument("--serve", type=int, default=40, help="requests of the serving sample (0: skip)")
    ap.add_argument("--profile-case", action="store_true", help="run the small ncu capture case and exit")
    ap.add_argument("--profile-ntt-group-mib", type=int, default=0,
                    help="profile case: NTT limb groups of at most this many MiB (0: whole sets)")
    ap.add_argument("--profile-modup-col", action="store_true",
                    help="profile case: the ModUp conversion inside the forward column pass")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch shapes")
    ap.add_argument("--large-argmin", type=int, default=0,
                    help="run only the blocked argmin of this many values on the n = 2^17 ring and exit")
    args = ap.parse_args()
    if args.large_argmin:
        return large_argmin(args.large_argmin)
    if args.profile_case:
        return profile_case(args.profile_ntt_group_mib, args.profile_modup_col)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_cuda(args)


if __name__ == "__main__":
    sys.exit(main())
