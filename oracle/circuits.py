"""The paper's circuits, step by step, over two oracle backends.

TEST INFRASTRUCTURE ONLY (imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py).

Backends:
  * ``PlainSlots`` - the noiseless model: a ciphertext is a float64 vector of the
    n/2 slots plus its level; a rotation is a cyclic shift, every polynomial is
    evaluated exactly.  It gives the ideal value of every intermediate.
  * ``OracleCkks`` - the same schedule on the plain RNS-CKKS of ``ckks.py``.

Slot layout (Sec. 2.3, row-by-row encoding): slot q*N^2 + i*N + j holds row i,
column j of the N x N matrix of query q (q = 0 .. Q-1 queries packed in one
ciphertext, Q*N^2 <= n/2).  A rotation amount r > 0 is a left rotation
(slot s <- slot s + r); r < 0 is a right rotation by -r.
"""
from __future__ import annotations

import math

import numpy as np

from . import ckks

# Cheon et al. composite sign polynomials (Sec. 2.2), coefficients of x, x^3, x^5, x^7.
F_COEFFS = (35 / 16, -35 / 16, 21 / 16, -5 / 16)
G_COEFFS = (4589 / 1024, -16577 / 1024, 25614 / 1024, -12860 / 1024)


def log2_exact(N: int) -> int:
    k = N.bit_length() - 1
    assert N == 1 << k, f"N={N} is not a power of two"
    return k


# --------------------------------------------------------------------------
# Plaintext masks (slot vectors)
# --------------------------------------------------------------------------
def mask_slots(kind: str, N: int, Q: int = 1, n_real: int | None = None, *, slots: int) -> np.ndarray:
    """Slot vector of a named plaintext, tiled over Q packed queries.
    n_real (<= N) is the unpadded length for the padding mask."""
    block = np.zeros((N, N))
    i, j = np.indices((N, N))
    if kind == "row0":            # MaskR(X, 0): keep row 0
        block[0, :] = 1.0
    elif kind == "col0":          # MaskC(X, 0): keep column 0
        block[:, 0] = 1.0
    elif kind == "tie":           # 4*delta_{j>=i} - 2 on the block (Alg. 6 folded, see rank_tie_corrected)
        block = np.where(j >= i, 2.0, -2.0)
    elif kind == "tri":           # delta_{j>=i}: upper triangle with the diagonal (Alg. 6)
        block = (j >= i).astype(float)
    elif kind == "row0s":         # MaskR(X, 0) scaled by 1/D: ranks leave SumR already divided by D
        block[0, :] = 1.0 / (N if n_real is None else n_real)     # D = the length ranks count
    elif kind == "col0s":         # MaskC(X, 0) scaled by 1/D
        block[:, 0] = 1.0 / (N if n_real is None else n_real)
    elif kind == "rowidx":        # -(a+1)/D in row a: Alg. 8's offset, less its block's constant
        block = -(i + 1.0) / (N if n_real is None else n_real)
    elif kind == "tiec":          # column form of "tie": 4*delta_{j<=i} - 2
        block = np.where(j <= i, 2.0, -2.0)
    elif kind == "sortidx":       # -(j+1)/N: column j of the sorting mask selects rank j+1 (Alg. 5)
        block = -(j + 1.0) / N
    elif kind == "valid":         # rows and columns of the unpadded vector (Sec. 3.1, padding)
        m = N if n_real is None else n_real
        block = ((i < m) & (j < m)).astype(float)
    else:
        raise ValueError(kind)
    v = np.zeros(slots)
    flat = block.reshape(-1)
    for q in range(Q):
        v[q * N * N:(q + 1) * N * N] = flat
    return v


# --------------------------------------------------------------------------
# Backends
# --------------------------------------------------------------------------
class PV:
    __slots__ = ("v", "level")

    def __init__(self, v, level):
        self.v = v
        self.level = level


class PlainSlots:
    """Noiseless slot model with level accounting (every product costs one level)."""

    def __init__(self, slots: int, top_level: int, radix2: bool = False):
        self.slots = slots
        self.top = top_level
        self.radix2 = radix2
        self.counts = {"rot": 0, "mul": 0, "mul_scalar": 0, "mul_plain": 0}

    def fresh(self, values) -> PV:
        v = np.zeros(self.slots)
        v[: len(values)] = values
        return PV(v, self.top)

    def level(self, x):
        return x.level

    def _lv(self, x, d=1):
        assert x.level - d >= 0, "out of levels"
        return x.level - d

    def rot(self, x, r):
        self.counts["rot"] += 1
        return PV(np.roll(x.v, -(r % self.slots)), x.level)

    def rot_many(self, x, rs):
        return [self.rot(x, r) for r in rs]

    def has_rot(self, r):
        """Whether a rotation by r is keyed (the model has every rotation unless told
        otherwise: `radix2` makes the chains take one doubling at a time)."""
        return not self.radix2

    def rot_sum(self, x, rs):
        self.counts["rot"] += len(rs)
        return PV(x.v + sum(np.roll(x.v, -(r % self.slots)) for r in rs), x.level)

    def add(self, x, y):
        assert x.level == y.level
        return PV(x.v + y.v, x.level)

    def sub(self, x, y):
        assert x.level == y.level
        return PV(x.v - y.v, x.level)

    def neg(self, x):
        return PV(-x.v, x.level)

    def mul(self, x, y):
        assert x.level == y.level
        self.counts["mul"] += 1
        return PV(x.v * y.v, self._lv(x))

    def mul_scalar(self, x, c):
        self.counts["mul_scalar"] += 1
        return PV(x.v * c, self._lv(x))

    def mul_plain(self, x, key):
        self.counts["mul_plain"] += 1
        return PV(x.v * mask_slots(*key, slots=self.slots), self._lv(x))

    def add_const(self, x, c):
        return PV(x.v + c, x.level)

    def add_plain(self, x, key):
        return PV(x.v + mask_slots(*key, slots=self.slots), x.level)

    def lincomb(self, xs, cs):
        assert all(x.level == xs[0].level for x in xs)
        self.counts["mul_scalar"] += 1
        return PV(sum(c * x.v for x, c in zip(xs, cs)), self._lv(xs[0]))

    def level_down(self, x, target):
        while x.level > target:
            x = self.mul_scalar(x, 1.0)
        return x

    def values(self, x):
        return x.v


class OracleCkks:
    """The schedule on the plain RNS-CKKS oracle."""

    def __init__(self, P: ckks.Params, keys: ckks.Keys):
        self.P = P
        self.keys = keys
        self.slots = P.slots
        self._enc = {}
        self.counts = {"rot": 0, "mul": 0, "mul_scalar": 0, "mul_plain": 0}

    def unscaled(self, key):
        if key not in self._enc:
            self._enc[key] = ckks.encode_unscaled(mask_slots(*key, slots=self.slots), self.P.n)
        return self._enc[key]

    def level(self, x):
        return x.level

    def rot(self, x, r):
        self.counts["rot"] += 1
        return ckks.rotate(self.P, self.keys, x, r)

    def rot_many(self, x, rs):
        return [self.rot(x, r) for r in rs]

    def has_rot(self, r):
        return ckks.galois_left(r % self.slots, self.P.n) in self.keys.gal

    def rot_sum(self, x, rs):
        self.counts["rot"] += len(rs)
        return ckks.rotate_sum(self.P, self.keys, x, rs)

    def add(self, x, y):
        return ckks.add(self.P, x, y)

    def sub(self, x, y):
        return ckks.sub(self.P, x, y)

    def neg(self, x):
        return ckks.neg(self.P, x)

    def mul(self, x, y):
        self.counts["mul"] += 1
        return ckks.mul(self.P, self.keys, x, y)

    def mul_scalar(self, x, c):
        self.counts["mul_scalar"] += 1
        return ckks.mul_scalar(self.P, x, c)

    def mul_plain(self, x, key):
        self.counts["mul_plain"] += 1
        return ckks.mul_plain(self.P, x, self.unscaled(key))

    def add_const(self, x, c):
        return ckks.add_const(self.P, x, c)

    def add_plain(self, x, key):
        return ckks.add_plain(self.P, x, self.unscaled(key))

    def lincomb(self, xs, cs):
        self.counts["mul_scalar"] += 1
        return ckks.lincomb(self.P, xs, cs)

    def level_down(self, x, target):
        return ckks.level_down(self.P, x, target)

    def values(self, x):
        return ckks.decrypt(self.P, self.keys, x)


# --------------------------------------------------------------------------
# Recursive matrix operations (App. A, Alg. 8-11; transpositions Alg. 1-2)
# --------------------------------------------------------------------------
def chain_pairs(B, amounts):
    """How a chain of doubling steps X <- X + (X << a_i) runs: consecutive steps
    (a_i, a_(i+1)) are taken two at a time as X + (X << a_i) + (X << a_(i+1)) +
    (X << a_i + a_(i+1)) with one hoisted ModUp and one ModDown (rot_sum) when the
    rotation by a_i + a_(i+1) is keyed; otherwise, and for a last odd step, one at a
    time.  Returns the list of steps, each a tuple of rotation amounts."""
    steps, i = [], 0
    while i < len(amounts):
        if i + 1 < len(amounts) and B.has_rot(amounts[i] + amounts[i + 1]):
            a, b = amounts[i], amounts[i + 1]
            steps.append((a, b, a + b))
            i += 2
        else:
            steps.append((amounts[i],))
            i += 1
    return steps


def steps_taken(step) -> int:
    """Doubling steps one entry of chain_pairs covers: two for (a, b, a + b), else one."""
    return 2 if len(step) > 1 else 1


def chain(B, x, amounts):
    """The doubling steps X <- X + (X << a) for a in amounts (left rotations; negative
    amounts rotate right), grouped as chain_pairs says."""
    for st in chain_pairs(B, amounts):
        x = B.rot_sum(x, list(st)) if len(st) > 1 else B.add(x, B.rot(x, st[0]))
    return x


def repl_r_amounts(N):
    return [-(N << i) for i in range(log2_exact(N))]


def trans_r_amounts(N):
    return [-((N * (N - 1)) >> i) for i in range(1, log2_exact(N) + 1)]


def repl_r(B, x, N):
    """Alg. 10: X <- X + (X >> N 2^i), i = 0 .. log N - 1."""
    return chain(B, x, repl_r_amounts(N))


def repl_c(B, x, N):
    """Alg. 11: X <- X + (X >> 2^i)."""
    return chain(B, x, [-(1 << i) for i in range(log2_exact(N))])


def sum_r(B, x, N, Q=1):
    """Alg. 8: X <- X + (X << N 2^i), then MaskR(X, 0)."""
    x = chain(B, x, [N << i for i in range(log2_exact(N))])
    return B.mul_plain(x, ("row0", N, Q))


def sum_c(B, x, N, Q=1):
    """Alg. 9: X <- X + (X << 2^i), then MaskC(X, 0)."""
    x = chain(B, x, [1 << i for i in range(log2_exact(N))])
    return B.mul_plain(x, ("col0", N, Q))


def trans_r(B, x, N, Q=1, trace=None):
    """Alg. 1: X <- X + (X >> N(N-1)/2^i), i = 1 .. log N, then MaskC(X, 0).  With a
    trace, one step at a time (the trace records every step)."""
    if trace is None:
        x = chain(B, x, trans_r_amounts(N))
    else:
        for r in trans_r_amounts(N):
            x = B.add(x, B.rot(x, r))
            trace.append((-r, x))
    return B.mul_plain(x, ("col0", N, Q))


def trans_c(B, x, N, Q=1, trace=None):
    """Alg. 2: X <- X + (X << N(N-1)/2^i), i = 1 .. log N, then MaskR(X, 0).  With a
    trace, one step at a time."""
    if trace is None:
        x = chain(B, x, [-r for r in trans_r_amounts(N)])
    else:
        for r in trans_r_amounts(N):
            x = B.add(x, B.rot(x, -r))
            trace.append((-r, x))
    return B.mul_plain(x, ("row0", N, Q))


# --------------------------------------------------------------------------
# Comparison (Sec. 2.2, composite f/g form)
# --------------------------------------------------------------------------
def poly7(B, x, c):
    """Odd degree-7 polynomial c1 x + c3 x^3 + c5 x^5 + c7 x^7 in multiplicative depth 3
    with four ciphertext products:  p = (c5 x + c7 x^3) x^4 + [(c3/c7)(c7 x^3) + c1 x],
    the bracket one exact linear combination (one rescale) of c7 x^3 and x brought down
    two levels; nine rescales in all."""
    c1, c3, c5, c7 = c
    y = B.mul(x, x)                                        # x^2          (l-1)
    z = B.mul(y, y)                                        # x^4          (l-2)
    x1 = B.mul_scalar(x, 1.0)                              # x            (l-1)
    b7 = B.mul(B.mul_scalar(x, c7), y)                     # c7 x^3       (l-2)
    a5 = B.mul_scalar(x1, c5)                              # c5 x         (l-2)
    hz = B.mul(B.add(a5, b7), z)                           # c5 x^5 + c7 x^7 (l-3)
    x2 = B.mul_scalar(x1, 1.0)                             # x            (l-2)
    rest = B.lincomb([b7, x2], [c3 / c7, c1])              # c3 x^3 + c1 x (l-3)
    return B.add(hz, rest)


def cmp_stages(dg: int, df: int):
    """g applied d_g times, then f applied d_f times; the last stage carries the 1/2 of
    Cmp = (f^df(g^dg(x)) + 1) / 2."""
    stages = [G_COEFFS] * dg + [F_COEFFS] * df
    out = []
    for idx, c in enumerate(stages):
        if idx == len(stages) - 1:
            c = tuple(ci / 2 for ci in c)
        out.append(c)
    return out


class ChebCmp:
    """The Chebyshev-approximated comparison (Sec. 2.2): the interpolant with `count`
    coefficients (first-kind nodes on [-1, 1]) of the step 1 (x > 0), 1/2 (x = 0),
    0 (x < 0), evaluated by Paterson-Stockmeyer; depth log2(count) + 1.  The step less
    1/2 is odd, so its even coefficients are zero: they are set to 0 exactly and the
    constant to 1/2, which keeps Cmp(x, x) = 1/2 exact.  Passed in place of d_g (d_f is
    then ignored) to every circuit below."""

    def __init__(self, count: int):
        assert count >= 4 and count & (count - 1) == 0
        self.count = count
        c = np.polynomial.chebyshev.chebinterpolate(
            lambda x: np.where(x > 0, 1.0, np.where(x < 0, 0.0, 0.5)), count - 1)
        c[2::2] = 0.0
        c[0] = 0.5
        self.coeffs = c

    def depth(self) -> int:
        return cheb_depth(self.count)


def cmp(B, x, dg, df):
    """Cmp(a, b) on x = a - b: 1 if a > b, 1/2 if equal, 0 if a < b (Eq. 1): the
    composite (f^d_f(g^d_g(x)) + 1)/2, or, with a ChebCmp in place of d_g, its
    Chebyshev approximation."""
    if isinstance(dg, ChebCmp):
        return cheb_ps(B, x, dg.coeffs)
    for c in cmp_stages(dg, df):
        x = poly7(B, x, c)
    return B.add_const(x, 0.5)


# --------------------------------------------------------------------------
# Ranking (Alg. 3) and tie correction (Alg. 6)
# --------------------------------------------------------------------------
def comparison_matrix(B, V, N, dg, df, Q=1):
    """C = Cmp(ReplR(V), ReplC(TransR(V))): slot iN+j holds Cmp(v_j, v_i) (Alg. 3 lines 1-3)."""
    VR, VC = row_col_forms(B, V, N, Q)
    return cmp(B, B.sub(VR, VC), dg, df)


def row_col_forms(B, V, N, Q=1):
    """V_R = ReplR(V) and V_C = ReplC(TransR(V)) (Alg. 3 lines 1-2), V_R brought down to
    V_C's level.  The first steps of ReplR and TransR both rotate V and share one
    ModUp (hoisting); each chain then runs as chain() groups it."""
    k = log2_exact(N)
    if k == 0:
        VR, VT = V, V
    else:
        ra, ta = repl_r_amounts(N), trans_r_amounts(N)
        r0, t0 = chain_pairs(B, ra)[0], chain_pairs(B, ta)[0]
        # the first step of each chain from V (one hoisted ModUp for both)
        if len(r0) == 1 and len(t0) == 1:
            r1, t1 = B.rot_many(V, [r0[0], t0[0]])
            VR, VT = B.add(V, r1), B.add(V, t1)
        else:
            step = lambda x, st: B.rot_sum(x, list(st)) if len(st) > 1 else B.add(x, B.rot(x, st[0]))
            VR, VT = step(V, r0), step(V, t0)
        VR = chain(B, VR, ra[steps_taken(r0):])
        VT = chain(B, VT, ta[steps_taken(t0):])
    T = B.mul_plain(VT, ("col0", N, Q))                     # TransR's MaskC
    VC = repl_c(B, T, N)
    return B.level_down(VR, B.level(VC)), VC


def rank_out_level(P, N) -> int:
    """Lowest level r whose modulus q_0 ... q_r holds ranks up to N at the canonical
    scale with two bits to spare: sum_i<=r log2 q_i >= log2 Delta_r + log2 N + 2."""
    bits = 0.0
    for r in range(P.L + 1):
        bits += math.log2(int(P.q[r]))
        if bits >= math.log2(P.scales[r]) + math.log2(N) + 2:
            return r
    return P.L


def cmp_levels(dg, df) -> int:
    """Levels one comparison consumes: 3 per composite stage (depth-3 degree-7
    polynomial), or the Chebyshev evaluation's depth."""
    return dg.depth() if isinstance(dg, ChebCmp) else 3 * (dg + df)


def rank(B, V, N, dg, df, Q=1, n_real=None, trim=False):
    """Alg. 3: R = SumR(C) + 1/2 (fractional ranks in row 0).  With n_real < N the
    vector was zero-padded to N = 2^k and the comparison matrix is masked to the
    n_real x n_real block before summing (Sec. 3.1).  trim: V is first brought down
    (level_down) to the lowest level the circuit needs, TransR's mask, the
    comparison, the padding mask and SumR's mask, so that the result leaves at
    level 0."""
    if trim:
        need = 1 + cmp_levels(dg, df) + 1 + (1 if n_real is not None and n_real != N else 0)
        V = B.level_down(V, need + rank_out_level(B.P, N))
    C = comparison_matrix(B, V, N, dg, df, Q)
    if n_real is not None and n_real != N:
        C = B.mul_plain(C, ("valid", N, Q, n_real))
    return B.add_const(sum_r(B, C, N, Q), 0.5)


def pack_tiles(B, xs, tile, per):
    """Pack ciphertexts whose slots outside [0, tile) are zero into groups of `per`:
    member k of a group moves to tile k (slots k tile + [0, tile)) by a tree of
    rotations (at step s = 1, 2, 4 ..: x_i += x_(i+s) >> s tile for every i whose
    place in its group is a multiple of 2s).  Returns one ciphertext per group."""
    xs = list(xs)
    m = len(xs)
    s = 1
    while s < per:
        for i in range(m):
            g = i % per
            if g % (2 * s) == 0 and g + s < per and i + s < m:
                xs[i] = B.add(xs[i], B.rot(xs[i + s], -tile * s))
        s *= 2
    return [xs[g * per] for g in range((m + per - 1) // per)]


def unpack_tiles(B, ys, counts, tile):
    """Inverse of pack_tiles: member k of group g is ys[g] rotated left by k tile (a
    tree: entry j + s = entry j << s tile), so its tile-0 slots hold what tile k held."""
    out = []
    for y, c in zip(ys, counts):
        part = [None] * c
        part[0] = y
        s = 1
        while s < c:
            for j in range(s):
                if j + s < c:
                    part[j + s] = B.rot(part[j], tile * s)
            s *= 2
        out += part
    return out


def packed_apply(B, xs, tile, per, f):
    """f on every x of xs, with the xs packed `per` to a ciphertext (per = 1: one by
    one): f must act slot by slot, and the xs must be zero outside [0, tile)."""
    if per <= 1:
        return [f(x) for x in xs]
    packed = pack_tiles(B, xs, tile, per)
    counts = [min(per, len(xs) - g * per) for g in range(len(packed))]
    return unpack_tiles(B, [f(p) for p in packed], counts, tile)


def rank_blocked(B, Vs, Bsz, dg, df, Q=1, pack=1):
    """Alg. 7, multi-ciphertext ranking of a vector split into L blocks of Bsz values
    (block i in row 0 of Vs[i]).  C_{i,j} = Cmp(ReplR(V_i), ReplC(TransR(V_j))) for
    j >= i only; by Eq. 3 the blocks j < i enter as 1 - C_{j,i}, summed column-wise
    and transposed:  R_i = TransC(SumC(sum_{j<i} (1 - C_{j,i}))) + SumR(sum_{j>=i} C_{i,j}) + 1/2.
    All R_i leave at the level of the TransC branch (SumR's branch is brought down).
    pack > 1: the comparisons run `pack` block pairs to a ciphertext (pairs in their
    listed order, i then j, packed into tiles of Q Bsz^2 slots by pack_tiles)."""
    L = len(Vs)
    forms = [row_col_forms(B, V, Bsz, Q) for V in Vs]
    pairs = [(i, j) for i in range(L) for j in range(i, L)]
    diffs = [B.sub(forms[i][0], forms[j][1]) for i, j in pairs]
    Cs = dict(zip(pairs, packed_apply(B, diffs, Q * Bsz * Bsz, pack, lambda x: cmp(B, x, dg, df))))
    out = []
    for i in range(L):
        A = Cs[(i, i)]
        for j in range(i + 1, L):
            A = B.add(A, Cs[(i, j)])
        S = sum_r(B, A, Bsz, Q)
        if i > 0:
            Bs = Cs[(0, i)]
            for j in range(1, i):
                Bs = B.add(Bs, Cs[(j, i)])
            T = trans_c(B, sum_c(B, B.add_const(B.neg(Bs), float(i)), Bsz, Q), Bsz, Q)
            R = B.add(B.level_down(S, B.level(T)), T)
        else:
            R = B.level_down(S, B.level(S) - 1)
        out.append(B.add_const(R, 0.5))
    return out


def cmp_strict(B, C):
    """Cmp_G = 2 C^2 - C: 1 where v_j > v_i, 0 at ties (Sec. 3.2, Min and Max)."""
    C2 = B.mul(C, C)
    return B.sub(B.add(C2, C2), B.level_down(C, B.level(C2)))


def rank_blocked_tc(B, Vs, Bsz, dg, df, Q=1, scaled=False, pack=1):
    """Tie-corrected multi-ciphertext ranking (Alg. 7 with Alg. 6): the rank of element
    b of block i counts the smaller elements and the equal ones at or before it in the
    global order (block i, position b).  Per block pair (Eq. 3 for j < i):
        j = i:  SumR(C_ii + E_ii (delta_{a<=b} - 1/2))  (the single-ciphertext fold)
        j > i:  SumR(G_ij)                 G = 2C^2 - C, strictly smaller elements of block j
        j < i:  TransC(SumC(1 - G_ji))     elements of block j not larger (all earlier ties count)
    scaled: every rank leaves divided by the total length D = L Bsz (masks 'row0s' with
    denominator D), the form the indicator of Alg. 4 and 8 takes.  pack > 1: the
    diagonal comparisons, and the upper ones with their Cmp_G, run `pack` to a
    ciphertext (pack_tiles).
    Returns the rank blocks (all at one level) and the ReplR forms of the blocks."""
    L = len(Vs)
    D = L * Bsz
    forms = [row_col_forms(B, V, Bsz, Q) for V in Vs]
    tile = Q * Bsz * Bsz
    diag = packed_apply(B, [B.sub(forms[i][0], forms[i][1]) for i in range(L)], tile, pack,
                        lambda x: cmp(B, x, dg, df))
    Cs = {(i, i): diag[i] for i in range(L)}
    upper = [(i, j) for i in range(L) for j in range(i + 1, L)]
    ups = packed_apply(B, [B.sub(forms[i][0], forms[j][1]) for i, j in upper], tile, pack,
                       lambda x: cmp_strict(B, cmp(B, x, dg, df)))
    Gs = dict(zip(upper, ups))
    rmask = ("row0s", Bsz, Q, D) if scaled else ("row0", Bsz, Q)
    out = []
    for i in range(L):
        A = tie_fold(B, Cs[(i, i)], Bsz, Q, "tie")
        for j in range(i + 1, L):
            A = B.add(A, B.level_down(Gs[(i, j)], B.level(A)))
        A = chain(B, A, [Bsz << r for r in range(log2_exact(Bsz))])
        S = B.mul_plain(A, rmask)
        if i > 0:
            Bs = Gs[(0, i)]
            for j in range(1, i):
                Bs = B.add(Bs, Gs[(j, i)])
            T = sum_c(B, B.add_const(B.neg(Bs), float(i)), Bsz, Q)
            T = chain(B, T, [-r for r in trans_r_amounts(Bsz)])
            T = B.mul_plain(T, rmask)
            S = B.add(S, B.level_down(T, B.level(S)))
        out.append(S)
    return out, [f[0] for f in forms]


def order_statistic_blocked(B, Vs, Bsz, k, dg, df, Q=1, coeffs=None, pack=1):
    """Alg. 4 over a multi-ciphertext vector: O_i = Ind_k(R_i) on the tie-corrected
    block ranks, one-hot at the first element of global rank k.  pack > 1: the block
    ranks (zero outside their tile) are packed before the constant -k/D is added, and
    the indicators run `pack` to a ciphertext."""
    D = len(Vs) * Bsz
    coeffs = sinc2_window_coeffs(D) if coeffs is None else coeffs
    Rs, _ = rank_blocked_tc(B, Vs, Bsz, dg, df, Q, scaled=True, pack=pack)
    return packed_apply(B, Rs, Q * Bsz * Bsz, pack, lambda R: cheb_ps(B, B.add_const(R, -k / D), coeffs))


def sort_blocked(B, Vs, Bsz, dg, df, Q=1, coeffs=None, pack=1):
    """Alg. 8 (multi-ciphertext sorting) on tie-corrected ranks:
        S_i = TransC(SumC(sum_j Ind_0(ReplR(R_j) - offset_i) . ReplR(V_j)))
    offset_i holds B i + a + 1 in row a (0-based block i): mask 'rowidx' plus the
    constant -B i / D, with ranks and offsets divided by D = L B.  pack > 1: the
    comparisons of the ranking and, per output block, its L indicators run `pack` to
    a ciphertext."""
    L = len(Vs)
    D = L * Bsz
    coeffs = sinc2_window_coeffs(D) if coeffs is None else coeffs
    Rs, VRs = rank_blocked_tc(B, Vs, Bsz, dg, df, Q, scaled=True, pack=pack)
    RR = [B.add_plain(repl_r(B, R, Bsz), ("rowidx", Bsz, Q, D)) for R in Rs]
    out = []
    for i in range(L):
        # the L indicators of output block i: RR_j (zero outside its tile) packed, then
        # the constant -B i / D, common to the group, added to every slot
        Ms = packed_apply(B, RR, Q * Bsz * Bsz, pack, lambda x: cheb_ps(B, B.add_const(x, -Bsz * i / D), coeffs))
        acc = None
        for j in range(L):
            M = Ms[j]
            P = B.mul(M, B.level_down(VRs[j], B.level(M)))
            acc = P if acc is None else B.add(acc, P)
        out.append(trans_c(B, sum_c(B, acc, Bsz, Q), Bsz, Q))
    return out


def tie_fold(B, C, N, Q=1, kind="tie"):
    """C + E (delta - 1/2) with E = 4 C (1 - C) = 4 K, K = C - C^2 (Alg. 6 before its
    SumR): the plaintext `kind` carries 4 delta - 2 (row form: delta_{j>=i}; column
    form 'tiec': delta_{j<=i})."""
    C2 = B.mul(C, C)
    Cd = B.level_down(C, B.level(C2))
    K = B.sub(Cd, C2)
    KT = B.mul_plain(K, (kind, N, Q))
    return B.add(B.level_down(Cd, B.level(KT)), KT)


def rank_tie_corrected(B, V, N, dg, df, Q=1):
    """Alg. 3 + Alg. 6 in one SumR:  R + F = SumR(C + E (delta_{j>=i} - 1/2)) with
    E = 4 C (1 - C);  the factor 4 and the -1/2 are folded into the 'tie' plaintext
    (4 delta - 2) applied to K = C - C^2.  The +1/2 of Alg. 3 and the -1/2 of Alg. 6 cancel."""
    C = comparison_matrix(B, V, N, dg, df, Q)
    return sum_r(B, tie_fold(B, C, N, Q, "tie"), N, Q)


# --------------------------------------------------------------------------
# Indicator: Chebyshev approximation evaluated by Paterson-Stockmeyer (Sec. 2.2)
# --------------------------------------------------------------------------
def sinc2_window_coeffs(N: int, degree: int | None = None) -> np.ndarray:
    """Chebyshev coefficients of the interpolant (first-kind nodes) on [-1, 1] of
    sinc^2(N t), degree max(8N, 128) - 1: 1 at t = 0 and 0 at every t = k/N, k != 0,
    so that p((r - k)/N) is the indicator Ind_k of Alg. 4 at integer ranks r."""
    d = max(8 * N, 128) - 1 if degree is None else degree
    return np.polynomial.chebyshev.chebinterpolate(lambda t: np.sinc(N * t) ** 2, d)


def baby_steps(length: int) -> int:
    """Number of baby steps k = 2^ceil(log2 sqrt(length)) for `length` coefficients."""
    k = 1 << math.ceil(math.log2(math.sqrt(length)))
    return min(k, length)


def cheb_ps(B, t, coeffs):
    """p(t) = sum_i c_i T_i(t) by Paterson-Stockmeyer in the Chebyshev basis.

    Baby steps T_1..T_k (T_2i = 2 T_i^2 - 1, T_2i+1 = 2 T_i T_i+1 - T_1), giant steps
    T_2m = 2 T_m^2 - 1 for m = k, 2k, ...; the coefficient vector (length a power of two,
    k * 2^j) is split recursively as p = q T_m + r with m half its length,
    q = c_m + sum_{j>=1} 2 c_{m+j} T_j and r = c_0 + sum_{i=1}^{m-1} (c_i - c_{2m-i}) T_i;
    a part of length k is a linear combination of T_1..T_{k-1} plus c_0.  Products
    bring both operands to the lower level first."""
    c = np.asarray(coeffs, dtype=np.float64)
    length = len(c)
    assert length >= 2 and length & (length - 1) == 0, "coefficient count must be a power of two"
    k = baby_steps(length)

    def prod2(a, b):  # 2 a b
        lo = min(B.level(a), B.level(b))
        y = B.mul(B.level_down(a, lo), B.level_down(b, lo))
        return B.add(y, y)

    T = {1: t}
    for i in range(2, k + 1):
        if i % 2 == 0:
            T[i] = B.add_const(prod2(T[i // 2], T[i // 2]), -1.0)
        else:
            y = prod2(T[i // 2], T[i // 2 + 1])
            T[i] = B.sub(y, B.level_down(T[1], B.level(y)))
    G = {k: T[k]}
    m = k
    while 2 * m < length:
        G[2 * m] = B.add_const(prod2(G[m], G[m]), -1.0)
        m *= 2
    leaf_level = min(B.level(T[i]) for i in range(1, k))
    TL = [B.level_down(T[i], leaf_level) for i in range(1, k)]

    def leaf(cc):
        return B.add_const(B.lincomb(TL, list(cc[1:])), float(cc[0]))

    def rec(cc):
        if len(cc) == k:
            return leaf(cc)
        m = len(cc) // 2
        q = np.empty(m)
        r = np.empty(m)
        q[0] = cc[m]
        q[1:] = 2.0 * cc[m + 1:]
        r[0] = cc[0]
        r[1:] = cc[1:m] - cc[2 * m - np.arange(1, m)]
        Qc = rec(q)
        Rc = rec(r)
        lo = min(B.level(Qc), B.level(G[m]))
        Pm = B.mul(B.level_down(Qc, lo), B.level_down(G[m], lo))
        return B.add(Pm, B.level_down(Rc, B.level(Pm)))

    return rec(c)


def cheb_depth(length: int) -> int:
    """Levels used by cheb_ps on `length` coefficients: log2(length) + 1."""
    return int(math.log2(length)) + 1


# --------------------------------------------------------------------------
# Order statistics (Alg. 4) and sorting (Alg. 5, column form)
# --------------------------------------------------------------------------
def sum_rows_masked(B, x, N, Q, kind):
    x = chain(B, x, [N << i for i in range(log2_exact(N))])
    return B.mul_plain(x, (kind, N, Q))


def sum_cols_masked(B, x, N, Q, kind):
    x = chain(B, x, [1 << i for i in range(log2_exact(N))])
    return B.mul_plain(x, (kind, N, Q))


def order_statistic(B, V, N, k, dg, df, Q=1, ties="first", coeffs=None):
    """O = Ind_k(R) (Alg. 4): a 0/1 row marking the element(s) of rank k.

    ties = "first": tie-corrected ranks (Alg. 6), one-hot at the first of equal
    elements.  ties = "all": k = 1 uses Cmp_G = 2C^2 - C (all minima rank 1),
    k = N uses Cmp_GE = 3C - 2C^2 (all maxima rank N) (Sec. 3.2, Min and Max);
    other k use the fractional ranks of Alg. 3.  The ranks leave SumR divided by N
    (mask 'row0s') and Ind_k(r) = p((r - k)/N) with p the sinc^2 window."""
    coeffs = sinc2_window_coeffs(N) if coeffs is None else coeffs
    if ties == "first":
        t = B.add_const(ranks_scaled_tc(B, V, N, dg, df, Q), -k / N)
        return cheb_ps(B, t, coeffs)
    C = comparison_matrix(B, V, N, dg, df, Q)
    if k == 1 or k == N:
        C2 = B.mul(C, C)
        Cd = B.level_down(C, B.level(C2))
        if k == 1:
            CG = B.sub(B.add(C2, C2), Cd)
            t = B.add_const(sum_rows_masked(B, CG, N, Q, "row0s"), (1.0 - k) / N)
        else:
            CG = B.sub(B.add(B.add(Cd, Cd), Cd), B.add(C2, C2))
            t = B.add_const(sum_rows_masked(B, CG, N, Q, "row0s"), -k / N)
    else:
        t = B.add_const(sum_rows_masked(B, C, N, Q, "row0s"), (0.5 - k) / N)
    return cheb_ps(B, t, coeffs)


def ranks_scaled_tc(B, V, N, dg, df, Q=1):
    """Tie-corrected ranks divided by N (Alg. 3 + Alg. 6, SumR with the mask 'row0s')."""
    C = comparison_matrix(B, V, N, dg, df, Q)
    return sum_rows_masked(B, tie_fold(B, C, N, Q, "tie"), N, Q, "row0s")


def order_value(B, V, N, k, dg, df, Q=1, coeffs=None):
    """The k-th smallest value (Alg. 4 with the value retrieval of Sec. 3.2):
    SumC(O . V) with O the tie-corrected one-hot mask, so that the division by the
    mask's L1 norm is by 1.  The value sits in slot 0 of each query (column 0 of row 0)."""
    O = order_statistic(B, V, N, k, dg, df, Q, "first", coeffs)
    return sum_c(B, B.mul(O, B.level_down(V, B.level(O))), N, Q)


def goldschmidt_iterations(N: int) -> int:
    """Iterations d of the inverse below for a mask weight m in [1, N]: the product
    prod_{i<=d} (1 + y^(2^i)) equals (1 - y^(2^(d+1))) / x for y = 1 - x, x = m / N, so its
    relative error is y^(2^(d+1)) <= (1 - 1/N)^(2^(d+1)); d is the smallest with that
    at most 2^-10."""
    d = 0
    while (1.0 - 1.0 / N) ** (2 ** (d + 1)) > 2.0 ** -10:
        d += 1
    return d


def inverse_goldschmidt(B, x, d):
    """1/x for slots x in (0, 1] by Goldschmidt's iteration: y = 1 - x, a = 1 + y,
    b = y^2, then d times a <- a (1 + b), b <- b^2 (one level each, the two products
    in parallel)."""
    y = B.add_const(B.neg(x), 1.0)
    a = B.add_const(y, 1.0)
    b = B.mul(y, y)
    a = B.level_down(a, B.level(b))
    for _ in range(d):
        a2 = B.mul(a, B.add_const(b, 1.0))
        b = B.mul(b, b)
        a = a2
    return a


def order_value_all(B, V, N, k, dg, df, Q=1, coeffs=None):
    """Value of the k-th order statistic from the all-ties mask (Sec. 3.2): O marks
    every element of rank k (k = 1: every minimum, Cmp_G; k = N: every maximum,
    Cmp_GE; other k: fractional ranks), and the value is <O, V> / |O|_1 =
    SumC(O . V) / SumC(O), the division by Goldschmidt's iteration on
    x = SumC(O) / N (goldschmidt_iterations(N) steps) with the 1/N folded into the
    numerator.  The value sits in slot 0 of each query; zero if no element has
    rank k."""
    O = order_statistic(B, V, N, k, dg, df, Q, "all", coeffs)
    num = sum_c(B, B.mul(O, B.level_down(V, B.level(O))), N, Q)
    den = sum_c(B, O, N, Q)
    x = B.mul_scalar(den, 1.0 / N)
    inv = inverse_goldschmidt(B, x, goldschmidt_iterations(N))
    numN = B.mul_scalar(num, 1.0 / N)
    lo = min(B.level(numN), B.level(inv))
    return B.mul(B.level_down(numN, lo), B.level_down(inv, lo))


def median(B, V, N, dg, df, Q=1, coeffs=None):
    """Median (Alg. 4's particular case): the (N+1)/2-th statistic for odd N, the mean of
    the N/2-th and (N/2+1)-th for even N, as SumC((O_a + O_b) . V/2) on one shared rank."""
    coeffs = sinc2_window_coeffs(N) if coeffs is None else coeffs
    R = ranks_scaled_tc(B, V, N, dg, df, Q)
    if N % 2:
        O = cheb_ps(B, B.add_const(R, -((N + 1) // 2) / N), coeffs)
        return sum_c(B, B.mul(O, B.level_down(V, B.level(O))), N, Q)
    Oa = cheb_ps(B, B.add_const(R, -(N // 2) / N), coeffs)
    Ob = cheb_ps(B, B.add_const(R, -(N // 2 + 1) / N), coeffs)
    M = B.add(Oa, Ob)
    Vh = B.mul_scalar(V, 0.5)
    return sum_c(B, B.mul(M, B.level_down(Vh, B.level(M))), N, Q)


def sort(B, V, N, dg, df, Q=1, coeffs=None):
    """Alg. 5 in column form (Sec. 3.3): ranks as a column, C' = Cmp(V_C, V_R),
    tie-corrected with 'tiec', SumC (scaled by 1/N), ReplC, minus (j+1)/N, the
    indicator around 0 gives M_ij = [r_i = j+1]; SumR(M . V_C) is the sorted row."""
    coeffs = sinc2_window_coeffs(N) if coeffs is None else coeffs
    VR, VC = row_col_forms(B, V, N, Q)
    Cc = cmp(B, B.sub(VC, VR), dg, df)
    S = sum_cols_masked(B, tie_fold(B, Cc, N, Q, "tiec"), N, Q, "col0s")
    D = B.add_plain(repl_c(B, S, N), ("sortidx", N, Q))
    M = cheb_ps(B, D, coeffs)
    Pm = B.mul(M, B.level_down(VC, B.level(M)))
    return sum_r(B, Pm, N, Q)


def tie_offset_unfolded(B, C, N, Q=1):
    """Alg. 6 as printed: E = 4 C (1 - C); U = SumR(E . delta_{j>=i}); T = SumR(E);
    F = U - T/2 - 1/2.  Used by the tests as the reference for the folded schedule."""
    E = B.mul_scalar(B.mul(C, B.add_const(B.neg(C), 1.0)), 4.0)
    U = sum_r(B, B.mul_plain(E, ("tri", N, Q)), N, Q)
    T = sum_r(B, B.level_down(E, B.level(E) - 1), N, Q)
    Th = B.mul_scalar(T, 0.5)
    F = B.add_const(B.sub(B.level_down(U, B.level(Th)), Th), -0.5)
    return E, U, T, F


# --------------------------------------------------------------------------
# Brute-force definitions (exact results the circuits approximate)
# --------------------------------------------------------------------------
def brute_fractional_rank(v):
    """r_j = #{i: v_i < v_j} + (#{i: v_i = v_j} + 1) / 2 (Sec. 3.1)."""
    v = np.asarray(v)
    less = (v[None, :] < v[:, None]).sum(axis=1)
    eq = (v[None, :] == v[:, None]).sum(axis=1)
    return less + 0.5 * (eq + 1)


def brute_tie_corrected_rank(v):
    """k_j = #{i: v_i < v_j} + #{i <= j: v_i = v_j} (Sec. 4): a stable sort's positions."""
    v = np.asarray(v)
    N = len(v)
    out = np.empty(N)
    for j in range(N):
        out[j] = np.sum(v < v[j]) + np.sum(v[: j + 1] == v[j])
    return out
