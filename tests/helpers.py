"""Shared test set-up: the parameter sets, the oracle's keys and encodings imported
into a CUDA context, and conversions between the two sides' formats."""
from __future__ import annotations

import numpy as np

from oracle import ckks, circuits

# name -> (log_n, n_limbs, log_q0, log_scale, n_special, log_special, digit_size, d_g, d_f)
CONFIGS = {
    "small": (11, 6, 60, 40, 2, 61, 2, 1, 1),
    "cfg1": (13, 14, 40, 40, 1, 61, 1, 2, 1),       # N = 8 rank, n = 2^13, 14 x ~40-bit + 1 special
    "cfg2": (16, 28, 60, 45, 3, 61, 3, 4, 2),       # N = 128 rank, n = 2^16, 28 limbs + 3 special
    "cfg3": (16, 34, 60, 45, 3, 61, 3, 3, 2),       # N = 128 ties, 34 limbs
    "ord": (11, 24, 60, 40, 2, 61, 2, 2, 1),        # deep small ring for order statistics / sort parity
    "ordb": (11, 24, 60, 40, 2, 61, 2, 1, 1),       # the same ring, shallower comparator: blocked sort parity
    # the smallest ring holding a 128 x 128 matrix, with the 34-limb chain of the tie
    # workload (not 128-bit secure at n = 2^15: a parity set only)
    "big15": (15, 34, 60, 45, 3, 61, 3, 3, 2),
    # a deeper n = 2^11 ring (test only): order statistics with the division of Sec. 3.2
    "deep": (11, 36, 60, 40, 3, 61, 3, 2, 1),
    # the n = 2^17 ring of the larger blocked order statistics and sorts, few limbs
    "ring17": (17, 8, 60, 40, 2, 61, 2, 1, 1),
    # a small ring whose primes are all k 2^32 + 1: every operation on that path
    "small_k32": (11, 6, 60, 45, 2, 61, 2, 1, 1),
}

# sets whose primes are all k 2^32 + 1 (prime_form 1; the others: = 1 mod 2n)
PRIME_FORM = {"cfg2": 1, "cfg3": 1, "big15": 1, "small_k32": 1}

MASK_IDS = {"row0": 1, "col0": 2, "tie": 3, "tri": 4, "valid": 5, "row0s": 6, "col0s": 7, "tiec": 8, "sortidx": 9,
            "rowidx": 10}
ALL_MASKS = ("row0", "col0", "tie", "tri", "row0s", "col0s", "tiec", "sortidx")


def oracle_params(name):
    log_n, n_limbs, log_q0, log_scale, alpha, log_sp, dsize, _, _ = CONFIGS[name]
    return ckks.gen_params(log_n, n_limbs, log_q0, log_scale, alpha, log_sp, dsize, PRIME_FORM.get(name, 0))


def gpu_context(name, device=0, cmp_cheb=0):
    from paper_2412_15126_gb300 import rankfhe
    log_n, n_limbs, log_q0, log_scale, alpha, log_sp, dsize, dg, df = CONFIGS[name]
    return rankfhe.Context(log_n, n_limbs, alpha, dsize, log_scale, log_q0, log_sp, dg, df, device=device,
                           cmp_cheb=cmp_cheb, prime_form=PRIME_FORM.get(name, 0))


def import_key(ctx, kind, g, key):
    """One oracle switching key: seeded keys travel as their b parts and the seed."""
    if key.seed is None:
        ctx.key_import(kind, g, key.data)
    else:
        ctx.key_import_seeded(kind, g, key.seed, key.data[:, 0])


def import_keys(ctx, keys):
    from paper_2412_15126_gb300 import rankfhe
    ctx.secret_import(keys.s)
    import_key(ctx, rankfhe.KEY_RELIN, 0, keys.rlk)
    for g, k in keys.gal.items():
        import_key(ctx, rankfhe.KEY_GALOIS, g, k)


def import_encodings(ctx, P, N, Q=1, n_real=None, kinds=("row0", "col0", "tie", "tri")):
    for kind in kinds:
        u = ckks.encode_unscaled(circuits.mask_slots(kind, N, Q, slots=P.slots), P.n)
        ctx.encoding_import(MASK_IDS[kind], N, Q, 0, u)
    if n_real is not None and n_real != N:
        u = ckks.encode_unscaled(circuits.mask_slots("valid", N, Q, n_real, slots=P.slots), P.n)
        ctx.encoding_import(MASK_IDS["valid"], N, Q, n_real, u)


def rotation_set(N, radix4=True):
    """Rotations of every circuit's chains for length N (ReplR, ReplC, SumR, SumC,
    TransR, TransC), and with radix4 the sums a_i + a_(i+1) of the step pairs the
    chains take two at a time (i = 0, 2, 4 ..)."""
    k = int(np.log2(N))
    rs = set()
    chains = [[-(N << i) for i in range(k)], [-(1 << i) for i in range(k)],
              [N << i for i in range(k)], [1 << i for i in range(k)],
              [-((N * (N - 1)) >> i) for i in range(1, k + 1)], [(N * (N - 1)) >> i for i in range(1, k + 1)]]
    for ch in chains:
        rs.update(ch)
        if radix4:
            rs.update(ch[i] + ch[i + 1] for i in range(0, len(ch) - 1, 2))
    return sorted(rs)


def galois_elts(P, rots):
    return sorted({ckks.galois_left(r % P.slots, P.n) for r in rots})
