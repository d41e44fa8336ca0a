"""GPU parity of the batched forms: stacked ciphertexts (one launch per kernel for
the stack) and slot packing (Q queries per ciphertext, masks tiled per query).

* Each member of a stacked rank is the oracle's rank of that input, bit for bit.
* rk_rank_batch on a mix of lengths returns, for every query, exactly the
  ciphertext its own rank returns alone.
* Slot-packed queries decrypt to their own brute-force ranks (no leakage).
"""
import numpy as np
import pytest

from oracle import ckks, circuits as C
from paper_2412_15126_gb300 import inputs
from tests import helpers

pytestmark = pytest.mark.gpu


def test_stacked_rank_bit_exact_per_member():
    P = helpers.oracle_params("cfg1")
    keys = ckks.keygen(P, 11, helpers.galois_elts(P, helpers.rotation_set(8)))
    ctx = helpers.gpu_context("cfg1")
    try:
        helpers.import_keys(ctx, keys)
        helpers.import_encodings(ctx, P, 8)
        vs = [inputs.gap_vector(8, 0.05, s) for s in (21, 22, 23)]
        cts = [ckks.encrypt(P, keys, v, s) for v, s in zip(vs, (21, 22, 23))]
        st = ctx.stack([ctx.ct_import(c.c, c.level, N=8) for c in cts])
        parts = ctx.unstack(ctx.rank(st))
        B = C.OracleCkks(P, keys)
        for ct, part, v in zip(cts, parts, vs):
            assert np.array_equal(part.export(), C.rank(B, ct, 8, 2, 1).c)
            assert np.max(np.abs(ctx.decrypt(part) - C.brute_fractional_rank(v))) < 0.25
    finally:
        ctx.close()


@pytest.fixture(scope="module")
def cfg2():
    ctx = helpers.gpu_context("cfg2")
    ctx.keygen(4242, 128)
    yield ctx
    ctx.close()


def test_rank_batch_identical_alone_and_in_mix(cfg2):
    ctx = cfg2
    lens = [16, 32, 16, 128, 64, 32, 128]
    vs = [inputs.gap_vector(N, 2.0 ** -9, 300 + i) for i, N in enumerate(lens)]
    cts = [ctx.encrypt(v, N=N) for v, N in zip(vs, lens)]
    mixed = ctx.rank_batch(cts)
    for ct, out, v in zip(cts, mixed, vs):
        alone = ctx.rank(ct)
        assert np.array_equal(out.export(), alone.export())
        assert np.max(np.abs(ctx.decrypt(out) - C.brute_fractional_rank(v))) < 0.25


def test_blocked_rank_bit_exact_n8x3():
    P = helpers.oracle_params("cfg1")
    keys = ckks.keygen(P, 12, helpers.galois_elts(P, helpers.rotation_set(8)))
    ctx = helpers.gpu_context("cfg1")
    try:
        helpers.import_keys(ctx, keys)
        helpers.import_encodings(ctx, P, 8)
        v = inputs.gap_vector(24, 0.04, 9)
        cts = [ckks.encrypt(P, keys, v[8 * i: 8 * i + 8], 40 + i) for i in range(3)]
        ref = C.rank_blocked(C.OracleCkks(P, keys), cts, 8, 2, 1)
        got = ctx.rank_blocked([ctx.ct_import(c.c, c.level, N=8) for c in cts])
        for g, r in zip(got, ref):
            assert np.array_equal(g.export(), r.c)
        ranks = np.concatenate([ctx.decrypt(g) for g in got])
        assert np.max(np.abs(ranks - C.brute_fractional_rank(v))) < 0.5
    finally:
        ctx.close()


def test_blocked_rank_n512(cfg2):
    ctx = cfg2
    v = inputs.gap_vector(512, 2.0 ** -9, 77)
    blocks = [ctx.encrypt(v[128 * i: 128 * (i + 1)], N=128) for i in range(4)]
    ranks = np.concatenate([ctx.decrypt(r) for r in ctx.rank_blocked(blocks)])
    assert np.max(np.abs(ranks - C.brute_fractional_rank(v))) < 0.25


@pytest.mark.parametrize("N,Q", [(16, 8), (32, 4), (64, 2)])
def test_slot_packed_queries(cfg2, N, Q):
    ctx = cfg2
    vs = [inputs.gap_vector(N, 2.0 ** -9, 500 + q) for q in range(Q)]
    ct = ctx.encrypt(np.concatenate(vs), N=N, Q=Q, n_real=N)
    got = ctx.decrypt(ctx.rank(ct)).reshape(Q, N)
    for q in range(Q):
        assert np.max(np.abs(got[q] - C.brute_fractional_rank(vs[q]))) < 0.25


@pytest.mark.parametrize("flags", [0, 1])
def test_graph_rank_bit_identical_to_direct(cfg2, flags):
    """The rank circuit captured as one CUDA graph replays to exactly the ciphertext
    the direct call returns, for fresh inputs of the captured shape (single and stacked)."""
    ctx = cfg2
    N = 32
    vs = [inputs.gap_vector(N, 2.0 ** -9, 500 + i) for i in range(5)]
    cts = [ctx.encrypt(v, N=N) for v in vs]
    g = ctx.graph_rank(cts[0], flags)
    try:
        for ct in cts[1:3]:                       # inputs other than the template
            assert np.array_equal(g.run(ct).export(), ctx.rank(ct, flags).export())
    finally:
        g.free()
    st = ctx.stack(cts[2:5])
    gs = ctx.graph_rank(st, flags)
    try:
        st2 = ctx.stack(cts[0:3])
        got = ctx.unstack(gs.run(st2))
        for ct, part in zip(cts[0:3], got):
            assert np.array_equal(part.export(), ctx.rank(ct, flags).export())
    finally:
        gs.free()


def test_order_stat_and_sort_batch_identical_alone():
    from paper_2412_15126_gb300 import rankfhe
    ctx = helpers.gpu_context("ord")
    try:
        ctx.keygen(66, 8)
        cts = [ctx.encrypt(inputs.grid_vector(N, 8, 40 + i), N=N) for i, N in enumerate((8, 4, 8, 8, 4))]
        for batch, alone in ((lambda c: ctx.order_stat_batch(c, 2, rankfhe.TIES_FIRST),
                              lambda x: ctx.order_stat(x, 2, rankfhe.TIES_FIRST)),
                             (lambda c: ctx.sort_batch(c), lambda x: ctx.sort(x))):
            for ct, out in zip(cts, batch(cts)):
                assert np.array_equal(out.export(), alone(ct).export())
    finally:
        ctx.close()


def _blob_records(blob):
    recs, at = {}, 5
    for _ in range(int(blob[4])):
        words = int(blob[at + 4])
        recs[(int(blob[at]), int(blob[at + 1]))] = (int(blob[at + 2]), int(blob[at + 3]), blob[at + 5: at + 5 + words])
        at += 5 + words
    assert at == blob.size
    return recs


@pytest.mark.parametrize("seeded", [True, False])
def test_keys_export_returns_the_imported_keys(seeded):
    """rk_keys_export gives back, word for word, the oracle's keys imported into the
    context (coefficient domain, plain residues: b parts and seeds for seeded keys,
    b and a otherwise), and importing the blob again changes no result."""
    P = helpers.oracle_params("small")
    keys = ckks.keygen(P, 17, helpers.galois_elts(P, [1, -1, 4]), seeded=seeded)
    ctx = helpers.gpu_context("small")
    try:
        helpers.import_keys(ctx, keys)
        blob = ctx.keys_export()
        assert int(blob[0]) == 0x32305359454B4B52 and int(blob[4]) == 1 + len(keys.gal)
        recs = _blob_records(blob)
        for kid, k in [((1, 0), keys.rlk)] + [((2, g), k) for g, k in keys.gal.items()]:
            flag, seed, words = recs[kid]
            assert flag == (1 if seeded else 0)
            want = k.data[:, 0] if seeded else k.data
            assert np.array_equal(words, np.asarray(want, dtype=np.uint64).reshape(-1))
            if seeded:
                assert seed == k.seed
        ct = ctx.encrypt(inputs.gap_vector(8, 0.05, 3), N=8)
        before = ctx.rotate(ct, 1).export()
        ctx.keys_import(blob)
        assert np.array_equal(ctx.rotate(ct, 1).export(), before)
    finally:
        ctx.close()


def test_explicit_and_seeded_keys_match_the_oracle():
    """The same circuit through explicit keys (a stored) and seeded keys (a regenerated
    inside the key switch): each bit-identical to the oracle with the same keys."""
    from oracle import circuits as C
    P = helpers.oracle_params("ordb")
    N = 8
    for seeded in (False, True):
        keys = ckks.keygen(P, 23, helpers.galois_elts(P, helpers.rotation_set(N)), seeded=seeded)
        ctx = helpers.gpu_context("ordb")
        try:
            helpers.import_keys(ctx, keys)
            helpers.import_encodings(ctx, P, N)
            ct = ckks.encrypt(P, keys, inputs.gap_vector(N, 0.05, 5), 31)
            ref = C.rank(C.OracleCkks(P, keys), ct, N, *helpers.CONFIGS["ordb"][7:9])
            got = ctx.rank(ctx.ct_import(ct.c, ct.level, N=N))
            assert np.array_equal(got.export(), ref.c)
        finally:
            ctx.close()


def test_graph_refuses_replay_after_scratch_growth(cfg2):
    """A captured graph points into the context's scratch: once a larger stack grows
    the scratch, replaying the old graph is refused (no access to freed memory)."""
    from paper_2412_15126_gb300 import rankfhe
    ctx = cfg2
    cts = [ctx.encrypt(inputs.gap_vector(32, 2.0 ** -9, 900 + i), N=32) for i in range(12)]
    g = ctx.graph_rank(cts[0])
    try:
        g.run(cts[1]).free()
        ctx.rank(ctx.stack(cts))          # twelve members: the scratch grows
        with pytest.raises(rankfhe.RkError):
            g.run(cts[2])
    finally:
        g.free()
    g2 = ctx.graph_rank(cts[0])           # a new capture works again
    try:
        assert np.array_equal(g2.run(cts[3]).export(), ctx.rank(cts[3]).export())
    finally:
        g2.free()


def test_graph_capture_every_circuit_bit_identical():
    """rk_graph_capture of the order statistic (a stack of two), the sort, and the
    blocked rank, order statistic and sort (two blocks of two queries each): every
    replay equals the direct call bit for bit, on inputs other than the template."""
    from paper_2412_15126_gb300 import rankfhe
    ctx = helpers.gpu_context("ordb")     # shallow comparator: the blocked sort of 2 x 4 fits 23 levels
    try:
        ctx.keygen(404, 8)
        mk = lambda s: ctx.encrypt(inputs.grid_vector(8, 16, s), N=8)
        pairs = [(ctx.stack([mk(1), mk(2)]), ctx.stack([mk(3), mk(4)])), (mk(5), mk(6))]
        cases = [
            (rankfhe.OP_ORDER_STAT, 1, rankfhe.TIES_FIRST, 1, pairs[0],
             lambda x: ctx.order_stat(x, 1, rankfhe.TIES_FIRST)),
            (rankfhe.OP_SORT, 0, 0, 1, pairs[1], lambda x: ctx.sort(x)),
        ]
        # blocked: block i of two queries is a stack of two; the template is the stack of
        # the L = 2 blocks, block-major
        q = [[ctx.encrypt(inputs.gap_vector(4, 0.05, 40 + 10 * a + b), N=4) for b in range(2)] for a in range(4)]
        blk = lambda a0, a1: [ctx.stack([q[a0][b], q[a1][b]]) for b in range(2)]
        tmpl_b, run_b = blk(0, 1), blk(2, 3)
        for op, direct in ((rankfhe.OP_RANK_BLOCKED, lambda bl: ctx.rank_blocked(bl)),
                           (rankfhe.OP_ORDER_STAT_BLOCKED, lambda bl: ctx.order_stat_blocked(bl, 3)),
                           (rankfhe.OP_SORT_BLOCKED, lambda bl: ctx.sort_blocked(bl))):
            g = ctx.graph_capture(op, ctx.stack(tmpl_b), arg=3 if op == rankfhe.OP_ORDER_STAT_BLOCKED else 0, L=2)
            got = ctx.unstack(g.run(ctx.stack(run_b)))
            want = [m for blk_out in direct(run_b) for m in ctx.unstack(blk_out)]
            assert len(got) == len(want) == 4
            for a, b in zip(got, want):
                assert np.array_equal(a.export(), b.export()), op
            g.free()
        for op, arg, flags, L, (tmpl, x), direct in cases:
            g = ctx.graph_capture(op, tmpl, arg=arg, flags=flags, L=L)
            got, want = g.run(x), direct(x)
            for a, b in zip(ctx.unstack(got), ctx.unstack(want)):
                assert np.array_equal(a.export(), b.export()), op
            g.free()
    finally:
        ctx.close()
