"""Pins of the tile packing of block-pair work (several B x B comparisons or indicator
evaluations in one ciphertext) in the noiseless slot model, against brute force and
against the unpacked circuits.

A B x B block fills B^2 of the n/2 slots; pack_tiles moves member k of a group to
slots k B^2 + [0, B^2) and unpack_tiles brings it back, so slot-wise work (the
comparator, the indicator) runs once per group instead of once per member.
"""
import numpy as np
import pytest

from oracle import circuits as C


def _blocks(B, v, Bsz):
    return [B.fresh(v[i * Bsz:(i + 1) * Bsz]) for i in range(len(v) // Bsz)]


@pytest.mark.parametrize("per, m", [(2, 3), (4, 4), (4, 7), (8, 5), (8, 16)])
def test_pack_then_unpack_restores_every_tile(per, m):
    """Packed tile k of group g holds member g per + k; unpacked member i holds, in its
    first tile, what member i held there; the members must be zero outside that tile."""
    tile = 16
    B = C.PlainSlots(tile * per, 5)
    rng = np.random.default_rng(per * 100 + m)
    data = [rng.uniform(-1, 1, tile) for _ in range(m)]
    xs = [B.fresh(d) for d in data]
    packed = C.pack_tiles(B, xs, tile, per)
    assert len(packed) == -(-m // per)
    for g, p in enumerate(packed):
        for k in range(per):
            i = g * per + k
            want = data[i] if i < m else np.zeros(tile)
            assert np.array_equal(B.values(p)[k * tile:(k + 1) * tile], want)
    counts = [min(per, m - g * per) for g in range(len(packed))]
    back = C.unpack_tiles(B, packed, counts, tile)
    assert len(back) == m
    for d, b in zip(data, back):
        assert np.array_equal(B.values(b)[:tile], d)
    # rotations: per - 1 a full group to pack and as many to unpack
    assert B.counts["rot"] == 2 * sum(c - 1 for c in counts)


@pytest.mark.parametrize("Bsz, L, per", [(4, 3, 2), (4, 3, 4), (2, 5, 8), (8, 2, 2)])
def test_packed_blocked_rank_is_the_rank(Bsz, L, per):
    """Alg. 7 with the block-pair comparisons packed per to a ciphertext gives the
    brute-force ranks and the unpacked circuit's row-0 values; the comparator runs on
    ceil(L(L+1)/2 / per) ciphertexts instead of L(L+1)/2."""
    rng = np.random.default_rng(Bsz * 7 + L + per)
    N = Bsz * L
    v = rng.permutation(np.linspace(0.01, 0.98, N))
    slots = per * Bsz * Bsz
    Bp = C.PlainSlots(slots, 40)
    Rp = C.rank_blocked(Bp, _blocks(Bp, v, Bsz), Bsz, 4, 2, pack=per)
    B1 = C.PlainSlots(slots, 40)
    R1 = C.rank_blocked(B1, _blocks(B1, v, Bsz), Bsz, 4, 2)
    got = np.concatenate([Bp.values(R)[:Bsz] for R in Rp])
    assert np.max(np.abs(got - C.brute_fractional_rank(v))) < 1e-3
    assert np.max(np.abs(got - np.concatenate([B1.values(R)[:Bsz] for R in R1]))) < 1e-12
    pairs = L * (L + 1) // 2
    assert Bp.counts["mul"] == -(-pairs // per) * 4 * 6 and B1.counts["mul"] == pairs * 4 * 6
    assert [R.level for R in Rp] == [R.level for R in R1]


@pytest.mark.parametrize("per", [2, 4])
def test_packed_blocked_tie_corrected_order_statistic_and_sort(per):
    """With ties across and within blocks: the stable ranks, the one-hot order
    statistic and the sorted vector, packed, equal brute force and the unpacked
    circuits' row-0 values."""
    Bsz, L = 4, 3
    v = np.array([5, 2, 9, 2, 7, 0, 5, 11, 0, 3, 9, 6]) / 24.0
    slots = per * Bsz * Bsz

    def run(f, pack):
        B = C.PlainSlots(slots, 80)
        out = f(B, _blocks(B, v, Bsz), pack)
        return np.concatenate([B.values(x)[:Bsz] for x in out]), [x.level for x in out]

    cases = [
        (lambda B, bl, p: C.rank_blocked_tc(B, bl, Bsz, 4, 2, pack=p)[0], C.brute_tie_corrected_rank(v)),
        (lambda B, bl, p: C.order_statistic_blocked(B, bl, Bsz, 3, 4, 2, pack=p),
         (C.brute_tie_corrected_rank(v) == 3).astype(float)),
        (lambda B, bl, p: C.sort_blocked(B, bl, Bsz, 4, 2, pack=p), np.sort(v)),
    ]
    for f, want in cases:
        got, lv = run(f, per)
        ref, lv1 = run(f, 1)
        assert np.max(np.abs(got - want)) < 1e-3
        assert np.max(np.abs(got - ref)) < 1e-9
        assert lv == lv1
