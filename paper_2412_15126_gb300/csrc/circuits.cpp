// The ranking circuits on the device evaluator.
//
// Slot layout (Sec. 2.3, row-by-row encoding): slot q N^2 + i N + j is row i,
// column j of packed query q.  A positive rotation amount is a left rotation.
// The schedule of every circuit below is fixed (it decides the exact ciphertext
// produced): matrix operations of App. A (Alg. 8-11) and Alg. 1, the composite
// comparison of Sec. 2.2, Alg. 3 for ranks and Alg. 6 for the tie offset.
#include <cmath>
#include <utility>

#include "rk_internal.cuh"

void mask_slot_values(uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real, size_t slots, std::vector<double>& v) {
    RK_REQUIRE((size_t)Q * N * N <= slots, RK_EINVAL, "mask does not fit the slots");
    v.assign(slots, 0.0);
    const uint32_t m = (kind == RK_MASK_VALID && n_real) ? n_real : N;
    for (uint32_t q = 0; q < Q; q++)
        for (uint32_t i = 0; i < N; i++)
            for (uint32_t j = 0; j < N; j++) {
                double x = 0.0;
                switch (kind) {
                    case RK_MASK_ROW0: x = i == 0 ? 1.0 : 0.0; break;
                    case RK_MASK_COL0: x = j == 0 ? 1.0 : 0.0; break;
                    case RK_MASK_TIE: x = j >= i ? 2.0 : -2.0; break;
                    case RK_MASK_TRI: x = j >= i ? 1.0 : 0.0; break;
                    case RK_MASK_VALID: x = (i < m && j < m) ? 1.0 : 0.0; break;
                    default: throw rk_error(RK_EINVAL, "unknown mask kind");
                }
                v[(size_t)q * N * N + (size_t)i * N + j] = x;
            }
}

namespace {

// Owning ciphertext handle for temporaries.
struct H {
    rk_ct* p = nullptr;
    H() = default;
    explicit H(rk_ct* x) : p(x) {}
    H(const H&) = delete;
    H& operator=(const H&) = delete;
    H(H&& o) noexcept : p(o.p) { o.p = nullptr; }
    H& operator=(H&& o) noexcept {
        if (this != &o) {
            if (p) ct_free(p);
            p = o.p;
            o.p = nullptr;
        }
        return *this;
    }
    ~H() {
        if (p) ct_free(p);
    }
    rk_ct* operator->() const { return p; }
    rk_ct* release() {
        rk_ct* t = p;
        p = nullptr;
        return t;
    }
};

struct Ev {
    rk_ctx* c;
    H fresh(const H& like, int level) { return H(ct_clone_meta(like.p, level)); }
    H copy(const H& x) {
        H o = fresh(x, x->level);
        ev_copy(c, x.p, o.p);
        return o;
    }
    H rot(const H& x, int r) {
        H o = fresh(x, x->level);
        rk_ct* outs[1] = {o.p};
        ev_rotate_many(c, x.p, &r, 1, outs);
        return o;
    }
    std::pair<H, H> rot2(const H& x, int r1, int r2) {
        H a = fresh(x, x->level), b = fresh(x, x->level);
        int r[2] = {r1, r2};
        rk_ct* outs[2] = {a.p, b.p};
        ev_rotate_many(c, x.p, r, 2, outs);
        return std::make_pair(std::move(a), std::move(b));
    }
    H add(const H& x, const H& y) {
        H o = fresh(x, x->level);
        ev_add(c, x.p, y.p, o.p);
        return o;
    }
    H sub(const H& x, const H& y) {
        H o = fresh(x, x->level);
        ev_sub(c, x.p, y.p, o.p);
        return o;
    }
    H mul(const H& x, const H& y) {
        H o = fresh(x, x->level);
        ev_mul(c, x.p, y.p, o.p);
        return o;
    }
    H mul_scalar(const H& x, double v) {
        H o = fresh(x, x->level);
        ev_mul_scalar(c, x.p, v, o.p);
        return o;
    }
    H mul_mask(const H& x, uint32_t kind) {
        H o = fresh(x, x->level);
        const uint32_t nr = kind == RK_MASK_VALID ? x->n_real : 0;
        ev_mul_plain(c, x.p, kind, x->N, x->Q, nr, o.p);
        return o;
    }
    H add_const(const H& x, double v) {
        H o = fresh(x, x->level);
        ev_add_const(c, x.p, v, o.p);
        return o;
    }
    H level_down(const H& x, int target) {
        H o = fresh(x, x->level);
        ev_level_down(c, x.p, target, o.p);
        return o;
    }
};

int log2_exact(uint32_t N) {
    int k = 0;
    while ((1u << k) < N) k++;
    RK_REQUIRE((1u << k) == N, RK_EINVAL, "N must be a power of two");
    return k;
}

// Cheon et al. composite sign polynomials (Sec. 2.2): coefficients of x, x^3, x^5, x^7.
const double kF[4] = {35.0 / 16, -35.0 / 16, 21.0 / 16, -5.0 / 16};
const double kG[4] = {4589.0 / 1024, -16577.0 / 1024, 25614.0 / 1024, -12860.0 / 1024};

// c1 x + c3 x^3 + c5 x^5 + c7 x^7 in depth 3 with four ciphertext products:
// p = (c5 x + c7 x^3) x^4 + (c3/c7)(c7 x^3) + c1 x.
H poly7(Ev& E, const H& x, const double c[4]) {
    const double c1 = c[0], c3 = c[1], c5 = c[2], c7 = c[3];
    H y = E.mul(x, x);
    H z = E.mul(y, y);
    H b7 = E.mul(E.mul_scalar(x, c7), y);
    H a5 = E.mul_scalar(E.mul_scalar(x, c5), 1.0);
    H hz = E.mul(E.add(a5, b7), z);
    H t3 = E.mul_scalar(b7, c3 / c7);
    H t1 = E.mul_scalar(E.mul_scalar(E.mul_scalar(x, c1), 1.0), 1.0);
    return E.add(E.add(hz, t3), t1);
}

// Cmp = (f^df(g^dg(x)) + 1) / 2 on x = a - b; the 1/2 rides on the last stage.
H cmp(Ev& E, H x, int dg, int df) {
    const int stages = dg + df;
    for (int s = 0; s < stages; s++) {
        const double* base = s < dg ? kG : kF;
        double c[4] = {base[0], base[1], base[2], base[3]};
        if (s == stages - 1)
            for (double& ci : c) ci /= 2;
        x = poly7(E, x, c);
    }
    return E.add_const(x, 0.5);
}

H sum_r(Ev& E, H x) {
    const int N = (int)x->N, k = log2_exact(x->N);
    for (int i = 0; i < k; i++) x = E.add(x, E.rot(x, N << i));
    return E.mul_mask(x, RK_MASK_ROW0);
}

// C = Cmp(ReplR(V), ReplC(TransR(V))); slot iN+j holds Cmp(v_j, v_i) (Alg. 3 lines 1-3).
H comparison_matrix(Ev& E, const H& V, int dg, int df) {
    const int N = (int)V->N, k = log2_exact(V->N);
    H VR, VT;
    if (k == 0) {
        VR = E.copy(V);
        VT = E.copy(V);
    } else {
        auto rt = E.rot2(V, -N, -((N * (N - 1)) >> 1));   // hoisted: one ModUp for both
        VR = E.add(V, rt.first);
        for (int i = 1; i < k; i++) VR = E.add(VR, E.rot(VR, -(N << i)));
        VT = E.add(V, rt.second);
        for (int i = 2; i <= k; i++) VT = E.add(VT, E.rot(VT, -((N * (N - 1)) >> i)));
    }
    H VC = E.mul_mask(VT, RK_MASK_COL0);                 // TransR's MaskC
    for (int i = 0; i < k; i++) VC = E.add(VC, E.rot(VC, -(1 << i)));
    H X = E.sub(E.level_down(VR, VC->level), VC);
    return cmp(E, std::move(X), dg, df);
}

}  // namespace

int rank_depth(const rk_ctx* c, const rk_ct* in, uint32_t flags) {
    int d = 1 + 3 * (int)(c->prm.d_g + c->prm.d_f) + 1;
    if (in->n_real != in->N) d += 1;
    if (flags & RK_TIES_CORRECT) d += 2;
    return d;
}

rk_ct* circuit_rank(rk_ctx* c, const rk_ct* in, uint32_t flags) {
    RK_REQUIRE(in->layout == RK_LAYOUT_ROW, RK_EINVAL, "rank expects a row vector");
    RK_REQUIRE((size_t)in->Q * in->N * in->N <= (size_t)c->n / 2, RK_EINVAL, "N^2 exceeds the slots");
    RK_REQUIRE(in->level >= rank_depth(c, in, flags), RK_EDEPTH,
               "rank needs " + std::to_string(rank_depth(c, in, flags)) + " levels, input has " + std::to_string(in->level));
    RK_REQUIRE(c->prm.d_g + c->prm.d_f >= 1, RK_EINVAL, "comparator needs at least one stage");
    RK_REQUIRE(!((flags & RK_TIES_CORRECT) && in->n_real != in->N), RK_EINVAL,
               "tie correction of a padded vector is not supported");
    Ev E{c};
    H V(ct_clone_meta(in, in->level));
    ev_copy(c, in, V.p);
    H C = comparison_matrix(E, V, (int)c->prm.d_g, (int)c->prm.d_f);
    if (in->n_real != in->N) C = E.mul_mask(C, RK_MASK_VALID);
    if (flags & RK_TIES_CORRECT) {
        // R + F = SumR(C + E (delta - 1/2)), E = 4 C (1 - C) = 4 K with K = C - C^2 (Alg. 6 folded)
        H C2 = E.mul(C, C);
        H Cd = E.level_down(C, C2->level);
        H K = E.sub(Cd, C2);
        H KT = E.mul_mask(K, RK_MASK_TIE);
        H W = E.add(E.level_down(Cd, KT->level), KT);
        return sum_r(E, std::move(W)).release();
    }
    H R = E.add_const(sum_r(E, std::move(C)), 0.5);
    return R.release();
}

rk_ct* circuit_compare_matrix(rk_ctx* c, const rk_ct* in) {
    RK_REQUIRE(in->layout == RK_LAYOUT_ROW, RK_EINVAL, "compare_matrix expects a row vector");
    RK_REQUIRE((size_t)in->Q * in->N * in->N <= (size_t)c->n / 2, RK_EINVAL, "N^2 exceeds the slots");
    const int need = 1 + 3 * (int)(c->prm.d_g + c->prm.d_f);
    RK_REQUIRE(in->level >= need, RK_EDEPTH, "comparison needs " + std::to_string(need) + " levels");
    RK_REQUIRE(c->prm.d_g + c->prm.d_f >= 1, RK_EINVAL, "comparator needs at least one stage");
    Ev E{c};
    H V(ct_clone_meta(in, in->level));
    ev_copy(c, in, V.p);
    return comparison_matrix(E, V, (int)c->prm.d_g, (int)c->prm.d_f).release();
}

// Rotation amounts the circuits use for a vector of length N (Sec. 3.1 and App. A).
void circuit_rotations(uint32_t N, std::vector<int>& out) {
    const int k = log2_exact(N);
    const int n = (int)N;
    for (int i = 0; i < k; i++) {
        out.push_back(-(n << i));   // ReplR
        out.push_back(n << i);      // SumR
        out.push_back(-(1 << i));   // ReplC
        out.push_back(1 << i);      // SumC
    }
    for (int i = 1; i <= k; i++) {
        out.push_back(-((n * (n - 1)) >> i));   // TransR
        out.push_back((n * (n - 1)) >> i);      // TransC
    }
}
