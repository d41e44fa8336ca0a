"""GPU parity: each homomorphic operation of the CUDA library, called through the
C-ABI on ciphertexts and keys made by the oracle, gives the oracle's ciphertext
bit for bit (canonical form: coefficient domain, residues in [0, q))."""
import numpy as np
import pytest

from oracle import ckks
from tests import helpers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["small", "cfg1", "small_k32"])
def setup(request):
    name = request.param
    P = helpers.oracle_params(name)
    rots = [1, 3, -1, -5, 17, P.slots // 2 - 1]
    keys = ckks.keygen(P, 77, helpers.galois_elts(P, rots))
    ctx = helpers.gpu_context(name)
    assert ctx.moduli() == list(P.q) + list(P.p)
    assert ctx.scales() == list(P.scales)
    helpers.import_keys(ctx, keys)
    rng = np.random.default_rng(3)
    z1 = rng.uniform(0, 1, P.slots)
    z2 = rng.uniform(0, 1, P.slots)
    c1 = ckks.encrypt(P, keys, z1, 1)
    c2 = ckks.encrypt(P, keys, z2, 2)
    g1 = ctx.ct_import(c1.c, c1.level)
    g2 = ctx.ct_import(c2.c, c2.level)
    yield P, keys, ctx, c1, c2, g1, g2, rots
    ctx.close()


def _same(gct, oct_):
    got = gct.export()
    assert got.shape == oct_.c.shape
    assert np.array_equal(got, oct_.c)


def test_import_export_round_trip(setup):
    P, keys, ctx, c1, c2, g1, g2, _ = setup
    _same(g1, c1)


def test_add_sub(setup):
    P, keys, ctx, c1, c2, g1, g2, _ = setup
    _same(ctx.add(g1, g2), ckks.add(P, c1, c2))
    _same(ctx.sub(g1, g2), ckks.sub(P, c1, c2))
    _same(ctx.add_const(g1, 0.3125), ckks.add_const(P, c1, 0.3125))


def test_rescale(setup):
    P, keys, ctx, c1, c2, g1, g2, _ = setup
    _same(ctx.rescale(g1), ckks.rescale(P, c1))


def test_mul_scalar(setup):
    P, keys, ctx, c1, c2, g1, g2, _ = setup
    for v in (1.0, -3.25, 25614 / 1024, 1e-3):
        _same(ctx.mul_scalar(g1, v), ckks.mul_scalar(P, c1, v))


def test_rotations(setup):
    P, keys, ctx, c1, c2, g1, g2, rots = setup
    for r in rots:
        _same(ctx.rotate(g1, r), ckks.rotate(P, keys, c1, r))


def test_hoisted_rotations_match_single(setup):
    P, keys, ctx, c1, c2, g1, g2, rots = setup
    outs = ctx.rotate_many(g1, rots[:3])
    for r, o in zip(rots[:3], outs):
        _same(o, ckks.rotate(P, keys, c1, r))


def test_mul_relin_rescale(setup):
    P, keys, ctx, c1, c2, g1, g2, _ = setup
    m = ckks.mul(P, keys, c1, c2)
    gm = ctx.mul(g1, g2)
    _same(gm, m)
    _same(ctx.mul(gm, gm), ckks.mul(P, keys, m, m))     # a lower level: truncated digits


def test_mul_mask(setup):
    P, keys, ctx, c1, c2, g1, g2, _ = setup
    N = 8
    helpers.import_encodings(ctx, P, N)
    g = ctx.ct_import(c1.c, c1.level, N=N)
    from oracle import circuits
    for kind in ("row0", "col0", "tie"):
        u = ckks.encode_unscaled(circuits.mask_slots(kind, N, 1, slots=P.slots), P.n)
        _same(ctx.mul_mask(g, helpers.MASK_IDS[kind]), ckks.mul_plain(P, c1, u))


def test_decrypt_matches_values(setup):
    P, keys, ctx, c1, c2, g1, g2, _ = setup
    z = ckks.decrypt(P, keys, c1)
    assert np.max(np.abs(ctx.decrypt_slots(g1) - z)) < 1e-9


def test_encrypt_on_gpu_decrypts(setup):
    P, keys, ctx, c1, c2, g1, g2, _ = setup
    v = np.linspace(0, 0.99, 8)
    g = ctx.encrypt(v, N=8)
    assert np.max(np.abs(ctx.decrypt(g) - v)) < 2.0 ** -20
    # the oracle decrypts the GPU's encryption under the same secret
    o = ckks.Ct(g.export(), g.level)
    assert np.max(np.abs(ckks.decrypt(P, keys, o)[:8] - v)) < 2.0 ** -20


def test_profile_pause_times_only_resumed_launches(setup):
    """rk_profile_pause: launches while paused are neither timed nor counted, the
    accumulators keep what was timed before, and results do not change."""
    P, keys, ctx, c1, c2, g1, g2, rots = setup
    ctx.profile_start("ks_inner")
    a = ctx.rotate(g1, rots[0])
    ctx.profile_pause(True)
    b = ctx.rotate(g1, rots[0])
    ctx.profile_pause(False)
    ctx.profile_stop()
    one = ctx.profile_kind("ks_inner")
    ctx.profile_start("ks_inner")
    ctx.rotate(g1, rots[0])
    ctx.profile_stop()
    alone = ctx.profile_kind("ks_inner")
    assert one["launches"] == alone["launches"] >= 1 and one["ms"] > 0
    assert one["bytes"] == alone["bytes"]
    assert np.array_equal(a.export(), b.export())
