"""GPU: the fused key-switching path (conversions inside the NTT passes, inner
product inside the row pass) against the staged one (lifted digits materialised),
bit for bit, for rotations (single and hoisted), products, stacked ciphertexts and
every L2 grouping of the lifted limbs.  The default path is the staged one; the
rotation / product parity tests elsewhere run it against the oracle, and
test_fused_path_matches_the_oracle runs the fused path against the oracle directly."""
import numpy as np
import pytest

from oracle import ckks
from paper_2412_15126_gb300 import inputs, rankfhe
from tests import helpers


def test_fused_path_matches_the_oracle():
    """With RK_OPT_KS_FUSED, a single rotation, a hoisted pair of rotations and a
    product equal the oracle's ciphertexts bit for bit (n = 2^13, 14 limbs)."""
    P = helpers.oracle_params("cfg1")
    rots = [-8, 3]
    keys = ckks.keygen(P, 19, helpers.galois_elts(P, rots))
    ctx = helpers.gpu_context("cfg1")
    try:
        helpers.import_keys(ctx, keys)
        ctx.set_option(rankfhe.OPT_KS_FUSED, 1)
        ct = ckks.encrypt(P, keys, inputs.gap_vector(8, 0.05, 19), 19)
        g = ctx.ct_import(ct.c, ct.level, N=8)
        assert np.array_equal(ctx.rotate(g, rots[0]).export(), ckks.rotate(P, keys, ct, rots[0]).c)
        for got, r in zip(ctx.rotate_many(g, rots), rots):
            assert np.array_equal(got.export(), ckks.rotate(P, keys, ct, r).c)
        assert np.array_equal(ctx.mul(g, g).export(), ckks.mul(P, keys, ct, ct).c)
    finally:
        ctx.close()

pytestmark = pytest.mark.gpu


def _run_ops(ctx, cts, rots):
    outs = []
    for ct in cts:
        outs += [ctx.rotate(ct, r).export() for r in rots]
        outs += [c.export() for c in ctx.rotate_many(ct, rots)]
        outs.append(ctx.mul(ct, ct).export())
    st = ctx.stack(cts)
    for part in ctx.unstack(ctx.rotate(st, rots[0])):
        outs.append(part.export())
    for part in ctx.unstack(ctx.mul(st, st)):
        outs.append(part.export())
    return outs


@pytest.mark.parametrize("name", ["small", "cfg1", "cfg2"])
def test_fused_equals_staged(name):
    ctx = helpers.gpu_context(name)
    try:
        N = 8
        ctx.keygen(77, N)
        rots = [1, 2, N, -1]
        ctx.keygen_rotations(rots)
        cts = [ctx.encrypt(inputs.gap_vector(N, 0.05, s), N=N) for s in (1, 2, 3)]
        ctx.set_option(rankfhe.OPT_KS_FUSED, 0)
        staged = _run_ops(ctx, cts, rots)
        ctx.set_option(rankfhe.OPT_KS_FUSED, 1)
        for group in (1, 3 << 20, 1 << 40):          # one limb a group .. every limb at once
            ctx.set_option(rankfhe.OPT_KS_GROUP_BYTES, group)
            fused = _run_ops(ctx, cts, rots)
            assert len(fused) == len(staged)
            for a, b in zip(fused, staged):
                assert np.array_equal(a, b)
    finally:
        ctx.close()


def test_set_option_rejects_unknown():
    ctx = helpers.gpu_context("small")
    try:
        with pytest.raises(rankfhe.RkError):
            ctx.set_option(99, 1)
        with pytest.raises(rankfhe.RkError):
            ctx.set_option(rankfhe.OPT_KS_GROUP_BYTES, -1)
    finally:
        ctx.close()


def test_autotune_keeps_results():
    """The autotuner changes launch shapes only: a rank is bit-identical before and after."""
    ctx = helpers.gpu_context("cfg1")
    try:
        ctx.keygen(3, 8)
        ct = ctx.encrypt(inputs.gap_vector(8, 0.05, 9), N=8)
        before = ctx.rank(ct).export()
        rep = ctx.autotune()
        assert rep["ntt_large_fwd_col"]["units"] >= 1 and rep["ntt_small_inv_row"]["us"] > 0
        assert rep["ntt_groups"]["us"]["whole"] > 0 and "ks" in rep
        after = ctx.rank(ct).export()
        assert np.array_equal(before, after)
    finally:
        ctx.close()


def test_ntt_limb_groups_keep_results():
    """NTTs run as limb groups (both passes of a group before the next) give the same
    words as one launch pair over the whole set: a rank on the n = 2^16, 28-limb set
    (whose top-level ModUp transforms 155 MB) with groups of 32 and 8 MiB."""
    ctx = helpers.gpu_context("cfg2")
    try:
        ctx.keygen(5, 128)
        ct = ctx.encrypt(inputs.gap_vector(128, 2.0 ** -9, 4), N=128)
        ctx.set_option(rankfhe.OPT_NTT_GROUP_BYTES, 0)
        whole = ctx.rank(ct).export()
        for mib in (32, 8):
            ctx.set_option(rankfhe.OPT_NTT_GROUP_BYTES, mib << 20)
            assert np.array_equal(ctx.rank(ct).export(), whole), mib
    finally:
        ctx.close()


@pytest.mark.parametrize("name, N", [("cfg1", 8), ("cfg2", 128)])
def test_modup_in_column_pass_keeps_results(name, N):
    """The staged key switch with the ModUp conversion inside the forward column pass
    (and the digits' own limbs copied by that kernel) gives the same rank, word for
    word, on a set with primes = 1 mod 2n and on one with primes k 2^32 + 1."""
    ctx = helpers.gpu_context(name)
    try:
        ctx.keygen(6, N)
        ct = ctx.encrypt(inputs.gap_vector(N, 2.0 ** -9 if N > 8 else 0.05, 5), N=N)
        staged = ctx.rank(ct).export()
        ctx.set_option(rankfhe.OPT_MODUP_COL, 1)
        assert np.array_equal(ctx.rank(ct).export(), staged)
    finally:
        ctx.close()


def test_fused_rank_equals_staged():
    """A whole rank (hoisted pair of rotations, the ReplR/TransR chains as one stack
    with a key per member, products with the single-rounding ModDown) through fused
    key switching equals the staged path bit for bit."""
    ctx = helpers.gpu_context("cfg1")
    try:
        ctx.keygen(31, 8)
        ct = ctx.encrypt(inputs.gap_vector(8, 0.05, 6), N=8)
        staged = ctx.rank(ct).export()
        ctx.set_option(rankfhe.OPT_KS_FUSED, 1)
        fused = ctx.rank(ct).export()
        ctx.set_option(rankfhe.OPT_KS_FUSED, 0)
        assert np.array_equal(staged, fused)
    finally:
        ctx.close()
