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
    const double D = n_real ? (double)n_real : (double)N;   // denominator of the scaled kinds
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
                    case RK_MASK_ROW0S: x = i == 0 ? 1.0 / D : 0.0; break;
                    case RK_MASK_COL0S: x = j == 0 ? 1.0 / D : 0.0; break;
                    case RK_MASK_TIEC: x = j <= i ? 2.0 : -2.0; break;
                    case RK_MASK_SORTIDX: x = -(j + 1.0) / N; break;
                    case RK_MASK_ROWIDX: x = -(i + 1.0) / D; break;
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
    H rot_add(const H& x, int r) {   // x + rot(x, r)
        H o = fresh(x, x->level);
        ev_rotate_add(c, x.p, r, o.p);
        return o;
    }
    H rot_add_multi(const H& x, const std::vector<int>& r) {   // member b: x_b + rot(x_b, r[b])
        H o = fresh(x, x->level);
        ev_rotate_multi(c, x.p, r.data(), true, o.p);
        return o;
    }
    // x_b + sum_k rot(x_b, r_b[k]) with one ModUp and one ModDown; r_b of one length
    // K <= 3 for every member b (member_r[b]), or the same list for all (one entry)
    H rot_sum(const H& x, const std::vector<std::vector<int>>& member_r) {
        const int B = x->B, K = (int)member_r[0].size();
        std::vector<int> r((size_t)3 * B, 0);
        for (int b = 0; b < B; b++) {
            const std::vector<int>& rb = member_r.size() == 1 ? member_r[0] : member_r[b];
            RK_REQUIRE((int)rb.size() == K, RK_EINVAL, "rot_sum: one rotation count for every member");
            for (int k = 0; k < K; k++) r[(size_t)b * 3 + k] = rb[k];
        }
        H o = fresh(x, x->level);
        rk_ct* outs[1] = {o.p};
        ev_rotate_sums(c, x.p, 1, &K, r.data(), true, outs);
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
    H mul_mask_d(const H& x, uint32_t kind, uint32_t D) {   // scaled kinds with denominator D
        H o = fresh(x, x->level);
        ev_mul_plain(c, x.p, kind, x->N, x->Q, D, o.p);
        return o;
    }
    H add_mask_d(const H& x, uint32_t kind, uint32_t D) {
        H o = fresh(x, x->level);
        ev_add_plain(c, x.p, kind, x->N, x->Q, D, o.p);
        return o;
    }
    H neg(const H& x) {
        H o = fresh(x, x->level);
        ev_neg(c, x.p, o.p);
        return o;
    }
    H add_const(const H& x, double v) {
        H o = fresh(x, x->level);
        ev_add_const(c, x.p, v, o.p);
        return o;
    }
    H add_mask(const H& x, uint32_t kind) {
        H o = fresh(x, x->level);
        ev_add_plain(c, x.p, kind, x->N, x->Q, 0, o.p);
        return o;
    }
    H lincomb(const std::vector<H>& xs, const double* cs) {
        std::vector<const rk_ct*> ps;
        std::vector<double> cv;
        for (size_t i = 0; i < xs.size(); i++) {
            ps.push_back(xs[i].p);
            cv.push_back(cs[i]);
        }
        H o = fresh(xs[0], xs[0]->level);
        ev_lincomb(c, ps, cv, o.p);
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

// Doubling chains X <- X + (X <<< a_i) (Alg. 1, 2, 8-11): consecutive steps are taken
// two at a time, X + (X <<< a_i) + (X <<< a_(i+1)) + (X <<< a_i + a_(i+1)) with one
// ModUp and one ModDown, when the rotation by a_i + a_(i+1) is keyed; otherwise, and
// for a last odd step, one at a time.  Each step is its list of rotation amounts.
bool has_rot(const rk_ctx* c, int r) {
    const u64 g = galois_left(c, r);
    return g != 1 && c->gal.count(g) > 0;
}
std::vector<std::vector<int>> chain_pairs(const rk_ctx* c, const std::vector<int>& a) {
    std::vector<std::vector<int>> steps;
    size_t i = 0;
    while (i < a.size()) {
        if (i + 1 < a.size() && has_rot(c, a[i] + a[i + 1])) {
            steps.push_back({a[i], a[i + 1], a[i] + a[i + 1]});
            i += 2;
        } else {
            steps.push_back({a[i]});
            i += 1;
        }
    }
    return steps;
}
int steps_taken(const std::vector<int>& step) { return step.size() > 1 ? 2 : 1; }

std::vector<int> repl_r_amounts(int N, int k) {
    std::vector<int> a;
    for (int i = 0; i < k; i++) a.push_back(-(N << i));
    return a;
}
std::vector<int> trans_r_amounts(int N, int k) {   // right rotations by N(N-1)/2^i, i = 1 .. k
    std::vector<int> a;
    for (int i = 1; i <= k; i++) a.push_back(-((N * (N - 1)) >> i));
    return a;
}
std::vector<int> pow2_amounts(int scale, int k, int sign) {   // sign scale 2^i, i < k
    std::vector<int> a;
    for (int i = 0; i < k; i++) a.push_back(sign * (scale << i));
    return a;
}
std::vector<int> negated(std::vector<int> a) {
    for (int& x : a) x = -x;
    return a;
}

// Cheon et al. composite sign polynomials (Sec. 2.2): coefficients of x, x^3, x^5, x^7.
const double kF[4] = {35.0 / 16, -35.0 / 16, 21.0 / 16, -5.0 / 16};
const double kG[4] = {4589.0 / 1024, -16577.0 / 1024, 25614.0 / 1024, -12860.0 / 1024};

// c1 x + c3 x^3 + c5 x^5 + c7 x^7 in depth 3 with four ciphertext products:
// p = (c5 x + c7 x^3) x^4 + [(c3/c7)(c7 x^3) + c1 x], the bracket one exact linear
// combination (one rescale) of c7 x^3 and x brought down two levels; nine rescales.
H poly7(Ev& E, const H& x, const double c[4]) {
    const double c1 = c[0], c3 = c[1], c5 = c[2], c7 = c[3];
    H y = E.mul(x, x);                        // x^2      (l-1)
    H x1 = E.mul_scalar(x, 1.0);              // x        (l-1)
    H c7x = E.mul_scalar(x, c7);              // c7 x     (l-1)
    H P, z, b7;                               // x^4, c7 x^3 (l-2)
    if (x->B <= 8) {
        // the two products of level l-1 as one stack of twice the members (no operand
        // copies); z and b7 are views into P, which outlives them
        const int B = x->B;
        const rk_ct* lhs[2] = {y.p, c7x.p};
        const rk_ct* rhs[2] = {y.p, y.p};
        P = H(ct_alloc_like(y.p, y->level, 2 * B));
        ev_mul_pairs(E.c, lhs, rhs, 2, P.p);
        z = H(ct_view_range(P.p, 0, B));
        b7 = H(ct_view_range(P.p, B, B));
    } else {
        z = E.mul(y, y);
        b7 = E.mul(c7x, y);
    }
    H a5 = E.mul_scalar(x1, c5);              // c5 x     (l-2)
    H hz = E.mul(E.add(a5, b7), z);           // c5 x^5 + c7 x^7 (l-3)
    H x2 = E.mul_scalar(x1, 1.0);             // x        (l-2)
    std::vector<H> terms;
    terms.push_back(std::move(b7));
    terms.push_back(std::move(x2));
    const double cs[2] = {c3 / c7, c1};
    H rest = E.lincomb(terms, cs);            // c3 x^3 + c1 x (l-3)
    return E.add(hz, rest);
}

H cheb_ps(Ev& E, const H& t, const std::vector<double>& c);
const std::vector<double>& cmp_cheb_coeffs(rk_ctx* c);

// Cmp = (f^df(g^dg(x)) + 1) / 2 on x = a - b; the 1/2 rides on the last stage.  A
// context with the Chebyshev comparator evaluates its interpolant instead (Sec. 2.2).
H cmp(Ev& E, H x, int dg, int df) {
    if (E.c->prm.cmp_cheb) return cheb_ps(E, x, cmp_cheb_coeffs(E.c));
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

// The chain's steps on x (every stack member by the same amounts).
H chain(Ev& E, H x, const std::vector<int>& amounts) {
    for (const auto& st : chain_pairs(E.c, amounts)) x = st.size() > 1 ? E.rot_sum(x, {st}) : E.rot_add(x, st[0]);
    return x;
}

// SumR (Alg. 8) with the row mask `kind` (RK_MASK_ROW0, or RK_MASK_ROW0S to divide by N)
H sum_rows(Ev& E, H x, uint32_t kind) {
    const int N = (int)x->N, k = log2_exact(x->N);
    x = chain(E, std::move(x), pow2_amounts(N, k, 1));
    return E.mul_mask(x, kind);
}
H sum_r(Ev& E, H x) { return sum_rows(E, std::move(x), RK_MASK_ROW0); }

// SumC (Alg. 9) with the column mask `kind`
H sum_cols(Ev& E, H x, uint32_t kind) {
    const int k = log2_exact(x->N);
    x = chain(E, std::move(x), pow2_amounts(1, k, 1));
    return E.mul_mask(x, kind);
}

// TransC (Alg. 2): X <- X + (X << N(N-1)/2^i), i = 1 .. log N, then MaskR(X, 0)
H trans_c(Ev& E, H x) {
    const int N = (int)x->N, k = log2_exact(x->N);
    x = chain(E, std::move(x), negated(trans_r_amounts(N, k)));
    return E.mul_mask(x, RK_MASK_ROW0);
}
// ReplC (Alg. 11)
H repl_c(Ev& E, H x) {
    const int k = log2_exact(x->N);
    return chain(E, std::move(x), pow2_amounts(1, k, -1));
}

// C + E (delta - 1/2), E = 4 K, K = C - C^2 (Alg. 6 before its SumR); the mask holds 4 delta - 2
H tie_fold(Ev& E, const H& C, uint32_t kind) {
    H C2 = E.mul(C, C);
    H Cd = E.level_down(C, C2->level);
    H K = E.sub(Cd, C2);
    H KT = E.mul_mask(K, kind);
    return E.add(E.level_down(Cd, KT->level), KT);
}

// 2 a b with both operands brought to the lower level first
H prod2(Ev& E, const H& a, const H& b) {
    const int lo = std::min(a->level, b->level);
    H y = E.mul(E.level_down(a, lo), E.level_down(b, lo));
    return E.add(y, y);
}

int baby_steps(int length) {
    int k = 1;
    while ((double)k * k < (double)length) k <<= 1;   // 2^ceil(log2 sqrt(length))
    return std::min(k, length);
}

// Products a_i * b_i (a_i and b_i of one level, all pairs of one level) as stacked
// products of up to 16 members: one launch per kernel and one key stream for a group.
// Each result is a view into its group's product, which `hold` keeps alive.
static std::vector<H> mul_group(Ev& E, const std::vector<const rk_ct*>& a, const std::vector<const rk_ct*>& b,
                                std::vector<H>& hold) {
    const int n = (int)a.size(), B = a[0]->B;
    const int per = std::max(1, 16 / B);
    std::vector<H> out;
    for (int g0 = 0; g0 < n; g0 += per) {
        const int g = std::min(per, n - g0);
        if (g == 1) {
            H o(ct_clone_meta(a[g0], a[g0]->level));
            ev_mul(E.c, a[g0], b[g0], o.p);
            out.push_back(std::move(o));
            continue;
        }
        H A(ct_stack(E.c, a.data() + g0, g)), Bs(ct_stack(E.c, b.data() + g0, g));
        H P = E.mul(A, Bs);
        for (int i = 0; i < g; i++) out.push_back(H(ct_view_range(P.p, i * B, B)));
        hold.push_back(std::move(P));
    }
    return out;
}

// p(t) = sum_i c_i T_i(t), Paterson-Stockmeyer in the Chebyshev basis: baby steps T_1..T_k,
// giant steps T_2m = 2 T_m^2 - 1; p = q T_m + r with m half the coefficient count,
// q = c_m + sum_{j>=1} 2 c_{m+j} T_j, r = c_0 + sum_{i=1}^{m-1} (c_i - c_{2m-i}) T_i; a part of
// k coefficients is sum_{i>=1} c_i T_i (one exact combination, one rescale) plus c_0.
// The baby steps of one doubling (T_{2^(w-1)+1} .. T_{2^w}) and the products of one depth
// of the split tree are independent: each group runs as stacked products.
struct ChebPS {
    Ev& E;
    int k;
    std::map<int, H> T, G;
    std::vector<H> TL;     // T_1..T_{k-1} at the leaf level
    std::vector<H> hold;   // stacked products the views point into
    struct Node {
        std::vector<double> cc;
        int q = -1, r = -1, depth = 0;
    };
    std::vector<Node> nodes;
    int build(const std::vector<double>& cc, int depth) {
        const int id = (int)nodes.size();
        nodes.push_back(Node{cc, -1, -1, depth});
        if ((int)cc.size() == k) return id;
        const int m = (int)cc.size() / 2;
        std::vector<double> q(m), r(m);
        q[0] = cc[m];
        for (int j = 1; j < m; j++) q[j] = 2.0 * cc[m + j];
        r[0] = cc[0];
        for (int i = 1; i < m; i++) r[i] = cc[i] - cc[2 * m - i];
        const int qi = build(q, depth + 1);
        const int ri = build(r, depth + 1);
        nodes[id].q = qi;
        nodes[id].r = ri;
        return id;
    }
    // depth first, one leaf at a time (little memory: for wide stacks)
    H rec(const std::vector<double>& cc) {
        if ((int)cc.size() == k) {
            H o = E.lincomb(TL, cc.data() + 1);
            return E.add_const(o, cc[0]);
        }
        const int m = (int)cc.size() / 2;
        std::vector<double> q(m), r(m);
        q[0] = cc[m];
        for (int j = 1; j < m; j++) q[j] = 2.0 * cc[m + j];
        r[0] = cc[0];
        for (int i = 1; i < m; i++) r[i] = cc[i] - cc[2 * m - i];
        H Qc = rec(q);
        H Rc = rec(r);
        const int lo = std::min(Qc->level, G[m]->level);
        H Pm = E.mul(E.level_down(Qc, lo), E.level_down(G[m], lo));
        return E.add(Pm, E.level_down(Rc, Pm->level));
    }
    // value of every node, deepest first: a node is Q T_m + R over its children (which
    // are released once used); all leaves are held at once, so this form is for stacks
    // of at most two members
    H eval(const std::vector<double>& c) {
        nodes.clear();
        build(c, 0);
        int deepest = 0;
        for (auto& nd : nodes) deepest = std::max(deepest, nd.depth);
        std::vector<H> val(nodes.size());
        // leaves: the combinations of T_1..T_{k-1} of a group land in the members of one
        // stack (up to 16 members), which takes one rescale; then each adds its c_0
        std::vector<int> leaves;
        for (size_t i = 0; i < nodes.size(); i++)
            if (nodes[i].q < 0) leaves.push_back((int)i);
        const int B = TL[0]->B, lvl = TL[0]->level;
        RK_REQUIRE(lvl >= 1, RK_EDEPTH, "Chebyshev leaves: no level left");
        std::vector<const rk_ct*> terms;
        for (auto& t : TL) terms.push_back(t.p);
        const int per = std::max(1, 16 / B), nl = (int)leaves.size();
        for (int j0 = 0; j0 < nl; j0 += per) {
            const int g = std::min(per, nl - j0);
            H Lst(ct_alloc_like(TL[0].p, lvl, g * B));
            for (int j = 0; j < g; j++) {
                H v(ct_view_range(Lst.p, j * B, B));
                const std::vector<double>& cc = nodes[leaves[j0 + j]].cc;
                ev_lincomb(E.c, terms, std::vector<double>(cc.begin() + 1, cc.end()), v.p, false);
            }
            Lst->level = lvl;
            ev_rescale_inplace(E.c, Lst.p);
            for (int j = 0; j < g; j++)
                val[leaves[j0 + j]] = E.add_const(H(ct_view_range(Lst.p, j * B, B)), nodes[leaves[j0 + j]].cc[0]);
        }
        for (int d = deepest - 1; d >= 0; d--) {
            std::vector<int> ids;
            for (size_t i = 0; i < nodes.size(); i++)
                if (nodes[i].depth == d && nodes[i].q >= 0) ids.push_back((int)i);
            if (ids.empty()) continue;
            const int m = (int)nodes[ids[0]].cc.size() / 2;
            std::vector<H> qs, gs;   // T_m brought down once per distinct level
            std::vector<const rk_ct*> a, b;
            for (int id : ids) {
                const H& Qc = val[nodes[id].q];
                const int lo = std::min(Qc->level, G[m]->level);
                qs.push_back(E.level_down(Qc, lo));
                if (gs.empty() || gs.back()->level != lo) gs.push_back(E.level_down(G[m], lo));
                a.push_back(qs.back().p);
                b.push_back(gs.back().p);
            }
            std::vector<H> prods = mul_group(E, a, b, hold);
            for (size_t i = 0; i < ids.size(); i++) {
                const H& Rc = val[nodes[ids[i]].r];
                val[ids[i]] = E.add(prods[i], E.level_down(Rc, prods[i]->level));
            }
            // this depth's operands and products are no longer needed
            for (int id : ids) {
                val[nodes[id].q] = H();
                val[nodes[id].r] = H();
            }
            prods.clear();
            qs.clear();
            gs.clear();
            hold.clear();
        }
        return std::move(val[0]);
    }
};

H cheb_ps(Ev& E, const H& t, const std::vector<double>& c) {
    const int length = (int)c.size();
    RK_REQUIRE(length >= 4 && (length & (length - 1)) == 0, RK_EINVAL, "Chebyshev coefficient count must be a power of two");
    ChebPS ps{E, baby_steps(length)};
    const int k = ps.k;
    ps.T[1] = E.copy(t);
    // baby steps by doubling: T_i for i in (w/2, w] from T_{i/2} and T_{i/2 + 1}, 2 a b
    // with both operands at the lower level (prod2)
    const int per = std::max(1, 16 / t->B);   // products a stacked group holds
    for (int w = 2; w <= k; w *= 2) {
        for (int i0 = w / 2 + 1; i0 <= w; i0 += per) {
            std::vector<H> ops, hold;
            std::vector<const rk_ct*> a, b;
            const int i1 = std::min(w, i0 + per - 1);
            for (int i = i0; i <= i1; i++) {
                const H& x = ps.T[i / 2];
                const H& y = ps.T[i % 2 == 0 ? i / 2 : i / 2 + 1];
                const int lo = std::min(x->level, y->level);
                ops.push_back(E.level_down(x, lo));
                a.push_back(ops.back().p);
                ops.push_back(E.level_down(y, lo));
                b.push_back(ops.back().p);
            }
            std::vector<H> prods = mul_group(E, a, b, hold);
            for (int i = i0; i <= i1; i++) {
                const H& p = prods[i - i0];
                H y2 = E.add(p, p);
                ps.T[i] = i % 2 == 0 ? E.add_const(y2, -1.0) : E.sub(y2, E.level_down(ps.T[1], y2->level));
            }
        }
    }
    ps.G[k] = E.copy(ps.T[k]);
    for (int m = k; 2 * m < length; m *= 2) ps.G[2 * m] = E.add_const(prod2(E, ps.G[m], ps.G[m]), -1.0);
    int leaf_level = 1 << 30;
    for (int i = 1; i < k; i++) leaf_level = std::min(leaf_level, ps.T[i]->level);
    for (int i = 1; i < k; i++) ps.TL.push_back(E.level_down(ps.T[i], leaf_level));
    ps.T.clear();   // the leaves and the giant steps hold everything the evaluation reads
    return t->B <= 2 ? ps.eval(c) : ps.rec(c);
}

int cheb_depth(int length) {
    int d = 0;
    while ((1 << d) < length) d++;
    return d + 1;
}

// Chebyshev coefficients (count of them) of the interpolant at the first-kind nodes on
// [-1, 1] of the step 1 (x > 0), 1/2 (x = 0), 0 (x < 0): the step less 1/2 is odd, so the
// even coefficients are set to 0 and the constant to 1/2 (Cmp(x, x) = 1/2 exactly).
std::vector<double> step_coeffs(int count) {
    std::vector<double> f(count), c(count);
    const double pi = 3.14159265358979323846;
    for (int kk = 0; kk < count; kk++) {
        const double x = std::cos(pi * (kk + 0.5) / count);
        f[kk] = x > 0 ? 1.0 : (x < 0 ? 0.0 : 0.5);
    }
    for (int j = 0; j < count; j++) {
        double acc = 0.0;
        for (int kk = 0; kk < count; kk++) acc += f[kk] * std::cos(j * pi * (kk + 0.5) / count);
        c[j] = (j % 2) ? 2.0 * acc / count : 0.0;
    }
    c[0] = 0.5;
    return c;
}

const std::vector<double>& cmp_cheb_coeffs(rk_ctx* c) {
    if (c->cmp_coeffs.empty()) c->cmp_coeffs = step_coeffs((int)c->prm.cmp_cheb);
    return c->cmp_coeffs;
}

// levels one comparison takes
int cmp_depth(const rk_ctx* c) {
    return c->prm.cmp_cheb ? cheb_depth((int)c->prm.cmp_cheb) : 3 * (int)(c->prm.d_g + c->prm.d_f);
}
bool cmp_ok(const rk_ctx* c) { return c->prm.cmp_cheb != 0 || c->prm.d_g + c->prm.d_f >= 1; }

// V_R = ReplR(V) and V_C = ReplC(TransR(V)) (Alg. 3 lines 1-2), V_R brought down to V_C's level.
std::pair<H, H> row_col_forms(Ev& E, const H& V) {
    const int N = (int)V->N, k = log2_exact(V->N);
    H VR, VT;
    if (k == 0) {
        VR = E.copy(V);
        VT = E.copy(V);
    } else {
        const std::vector<int> ra = repl_r_amounts(N, k), ta = trans_r_amounts(N, k);
        const std::vector<int> r0 = chain_pairs(E.c, ra)[0], t0 = chain_pairs(E.c, ta)[0];
        if (r0.size() == 1 && t0.size() == 1) {
            auto rt = E.rot2(V, r0[0], t0[0]);   // hoisted: one ModUp for both
            VR = E.add(V, rt.first);
            VT = E.add(V, rt.second);
        } else {   // both chains' first steps from V: one ModUp, one ModDown
            VR = E.fresh(V, V->level);
            VT = E.fresh(V, V->level);
            const int B = V->B;
            const int K[2] = {(int)r0.size(), (int)t0.size()};
            std::vector<int> r((size_t)2 * B * 3, 0);
            for (int b = 0; b < B; b++)
                for (int j = 0; j < 3; j++) {
                    if (j < K[0]) r[(size_t)b * 3 + j] = r0[j];
                    if (j < K[1]) r[((size_t)B + b) * 3 + j] = t0[j];
                }
            rk_ct* outs[2] = {VR.p, VT.p};
            ev_rotate_sums(E.c, V.p, 2, K, r.data(), true, outs);
        }
        const std::vector<int> rrest(ra.begin() + steps_taken(r0), ra.end()), trest(ta.begin() + steps_taken(t0), ta.end());
        const auto rs = chain_pairs(E.c, rrest), ts = chain_pairs(E.c, trest);
        bool lockstep = V->B == 1 && !rs.empty() && rs.size() == ts.size();
        for (size_t i = 0; lockstep && i < rs.size(); i++) lockstep = rs[i].size() == ts[i].size();
        if (lockstep) {
            // the two chains in step, as one two-member stack with a key per member
            const rk_ct* pair[2] = {VR.p, VT.p};
            H S(ct_stack(E.c, pair, 2));
            for (size_t i = 0; i < rs.size(); i++)
                S = rs[i].size() > 1 ? E.rot_sum(S, {rs[i], ts[i]}) : E.rot_add_multi(S, {rs[i][0], ts[i][0]});
            VR = E.copy(H(ct_view(S.p, 0)));
            VT = E.copy(H(ct_view(S.p, 1)));
        } else {
            VR = chain(E, std::move(VR), rrest);
            VT = chain(E, std::move(VT), trest);
        }
    }
    H VC = E.mul_mask(VT, RK_MASK_COL0);                 // TransR's MaskC
    VC = repl_c(E, std::move(VC));
    H VRd = E.level_down(VR, VC->level);
    return std::make_pair(std::move(VRd), std::move(VC));
}

// C = Cmp(ReplR(V), ReplC(TransR(V))); slot iN+j holds Cmp(v_j, v_i) (Alg. 3 lines 1-3).
H comparison_matrix(Ev& E, const H& V, int dg, int df) {
    auto rc = row_col_forms(E, V);
    return cmp(E, E.sub(rc.first, rc.second), dg, df);
}

// Chebyshev coefficients of the interpolant of sinc^2(N t) on [-1, 1] at the count
// Chebyshev nodes of the first kind: c_j = (2/count) sum_k f(x_k) cos(j theta_k), c_0 halved.
std::vector<double> sinc2_coeffs(uint32_t N, int count) {
    std::vector<double> f(count), c(count);
    const double pi = 3.14159265358979323846;
    for (int kk = 0; kk < count; kk++) {
        const double th = pi * (kk + 0.5) / count;
        const double x = N * std::cos(th);
        const double s = x == 0.0 ? 1.0 : std::sin(pi * x) / (pi * x);
        f[kk] = s * s;
    }
    for (int j = 0; j < count; j++) {
        double acc = 0.0;
        for (int kk = 0; kk < count; kk++) acc += f[kk] * std::cos(j * pi * (kk + 0.5) / count);
        c[j] = 2.0 * acc / count;
    }
    c[0] *= 0.5;
    return c;
}

const std::vector<double>& indicator_coeffs(rk_ctx* c, uint32_t N) {
    auto it = c->indicator.find(N);
    if (it == c->indicator.end()) it = c->indicator.emplace(N, sinc2_coeffs(N, std::max(8 * (int)N, 128))).first;
    return it->second;
}

}  // namespace

// Lowest level r whose modulus q_0 .. q_r holds ranks up to N at the canonical scale
// with two bits to spare: where a trimmed rank leaves (q_0 of 40 bits at scale 2^40
// cannot hold the 1/2 the rank adds to every slot).
static int rank_out_level(const rk_ctx* c, uint32_t N) {
    double bits = 0.0;
    for (int r = 0; r <= c->L; r++) {
        bits += std::log2((double)c->primes[r]);
        if (bits >= std::log2(c->scales[r]) + std::log2((double)N) + 2.0) return r;
    }
    return c->L;
}

// levels the rank circuit consumes
int rank_depth(const rk_ctx* c, const rk_ct* in, uint32_t flags) {
    int d = 1 + cmp_depth(c) + 1;
    if (in->n_real != in->N) d += 1;
    if (flags & RK_TIES_CORRECT) d += 2;
    return d;
}

rk_ct* circuit_rank(rk_ctx* c, const rk_ct* in, uint32_t flags) {
    RK_REQUIRE(in->layout == RK_LAYOUT_ROW, RK_EINVAL, "rank expects a row vector");
    RK_REQUIRE((size_t)in->Q * in->N * in->N <= (size_t)c->n / 2, RK_EINVAL, "N^2 exceeds the slots");
    RK_REQUIRE(in->level >= rank_depth(c, in, flags), RK_EDEPTH,
               "rank needs " + std::to_string(rank_depth(c, in, flags)) + " levels, input has " + std::to_string(in->level));
    RK_REQUIRE(cmp_ok(c), RK_EINVAL, "comparator needs at least one stage");
    RK_REQUIRE(!((flags & RK_TIES_CORRECT) && in->n_real != in->N), RK_EINVAL,
               "tie correction of a padded vector is not supported");
    Ev E{c};
    H V(ct_clone_meta(in, in->level));
    ev_copy(c, in, V.p);
    const int keep = rank_depth(c, in, flags) + rank_out_level(c, in->N);
    if (c->trim_levels && V->level > keep) V = E.level_down(V, keep);   // the result leaves at rank_out_level
    H C = comparison_matrix(E, V, (int)c->prm.d_g, (int)c->prm.d_f);
    if (in->n_real != in->N) C = E.mul_mask(C, RK_MASK_VALID);
    if (flags & RK_TIES_CORRECT)   // R + F = SumR(C + E (delta - 1/2)) (Alg. 6 folded)
        return sum_r(E, tie_fold(E, C, RK_MASK_TIE)).release();
    H R = E.add_const(sum_r(E, std::move(C)), 0.5);
    return R.release();
}

const std::vector<double>& indicator_coeffs_of(rk_ctx* c, uint32_t N) { return indicator_coeffs(c, N); }
const std::vector<double>& comparator_coeffs_of(rk_ctx* c) {
    RK_REQUIRE(c->prm.cmp_cheb != 0, RK_EINVAL, "the context uses the composite comparator (no Chebyshev coefficients)");
    return cmp_cheb_coeffs(c);
}

void indicator_import(rk_ctx* c, uint32_t N, const double* coeffs, size_t count) {
    RK_REQUIRE(count >= 4 && (count & (count - 1)) == 0, RK_EINVAL, "coefficient count must be a power of two >= 4");
    c->indicator[N] = std::vector<double>(coeffs, coeffs + count);
    c->generation++;
}

static void check_square(rk_ctx* c, const rk_ct* in, int need, const char* what) {
    RK_REQUIRE(in->layout == RK_LAYOUT_ROW, RK_EINVAL, std::string(what) + " expects a row vector");
    RK_REQUIRE((size_t)in->Q * in->N * in->N <= (size_t)c->n / 2, RK_EINVAL, "N^2 exceeds the slots");
    RK_REQUIRE(in->n_real == in->N, RK_EINVAL, std::string(what) + " of a padded vector is not supported");
    RK_REQUIRE(cmp_ok(c), RK_EINVAL, "comparator needs at least one stage");
    RK_REQUIRE(in->level >= need, RK_EDEPTH,
               std::string(what) + " needs " + std::to_string(need) + " levels, input has " + std::to_string(in->level));
}

int order_stat_depth(rk_ctx* c, const rk_ct* in, uint32_t k, uint32_t flags) {
    const int dc = cmp_depth(c);
    const int ind = cheb_depth((int)indicator_coeffs(c, in->N).size());
    int extra = 0;
    if (!(flags & RK_TIES_ALL)) extra = 2;                              // tie fold
    else if (k == 1 || k == in->N) extra = 1;                           // Cmp_G / Cmp_GE
    return 1 + dc + extra + 1 + ind;
}

// Alg. 4: O = Ind_k(R), ranks leaving SumR divided by N, Ind_k(r) = p((r - k)/N).
rk_ct* circuit_order_stat(rk_ctx* c, const rk_ct* in, uint32_t k, uint32_t flags) {
    RK_REQUIRE(k >= 1 && k <= in->N, RK_EINVAL, "k must be in [1, N]");
    check_square(c, in, order_stat_depth(c, in, k, flags), "order statistic");
    const double N = (double)in->N;
    Ev E{c};
    H V(ct_clone_meta(in, in->level));
    ev_copy(c, in, V.p);
    H C = comparison_matrix(E, V, (int)c->prm.d_g, (int)c->prm.d_f);
    H t;
    if (!(flags & RK_TIES_ALL)) {
        t = E.add_const(sum_rows(E, tie_fold(E, C, RK_MASK_TIE), RK_MASK_ROW0S), -(double)k / N);
    } else if (k == 1 || k == in->N) {
        H C2 = E.mul(C, C);
        H Cd = E.level_down(C, C2->level);
        if (k == 1) {   // Cmp_G = 2 C^2 - C: every minimum has rank 1
            H CG = E.sub(E.add(C2, C2), Cd);
            t = E.add_const(sum_rows(E, std::move(CG), RK_MASK_ROW0S), (1.0 - (double)k) / N);
        } else {        // Cmp_GE = 3 C - 2 C^2: every maximum has rank N
            H CG = E.sub(E.add(E.add(Cd, Cd), Cd), E.add(C2, C2));
            t = E.add_const(sum_rows(E, std::move(CG), RK_MASK_ROW0S), -(double)k / N);
        }
    } else {
        t = E.add_const(sum_rows(E, std::move(C), RK_MASK_ROW0S), (0.5 - (double)k) / N);
    }
    return cheb_ps(E, t, indicator_coeffs(c, in->N)).release();
}

static H stack_of(rk_ctx* c, const std::vector<rk_ct*>& xs);
static H range(const H& st, int i, int Bq);

int order_value_depth(rk_ctx* c, const rk_ct* in) { return order_stat_depth(c, in, 1, RK_TIES_FIRST) + 2; }

// The k-th smallest value (Alg. 4 with the value retrieval of Sec. 3.2): SumC(O . V),
// O the tie-corrected one-hot mask (its L1 norm is 1, so no division); the value is in
// slot 0 of each query (column 0 of row 0; SumC's mask clears the other columns).
rk_ct* circuit_order_value(rk_ctx* c, const rk_ct* in, uint32_t k) {
    check_square(c, in, order_value_depth(c, in), "order value");
    Ev E{c};
    H O(circuit_order_stat(c, in, k, RK_TIES_FIRST));
    H V(ct_clone_meta(in, in->level));
    ev_copy(c, in, V.p);
    return sum_cols(E, E.mul(O, E.level_down(V, O->level)), RK_MASK_COL0).release();
}

// Iterations of the Goldschmidt inverse for a mask weight in [1, N]: the smallest d with
// (1 - 1/N)^(2^(d+1)) <= 2^-10 (the relative error of prod_{i<=d} (1 + y^(2^i)) as 1/x).
static int goldschmidt_iterations(uint32_t N) {
    int d = 0;
    while (std::pow(1.0 - 1.0 / (double)N, std::pow(2.0, d + 1)) > std::pow(2.0, -10)) d++;
    return d;
}

int order_value_all_depth(rk_ctx* c, const rk_ct* in, uint32_t k) {
    // O, then SumC (mask), the 1/N scalar, y^2, d iterations and the final product
    return order_stat_depth(c, in, k, RK_TIES_ALL) + 4 + goldschmidt_iterations(in->N);
}

// The value of the k-th statistic from the all-ties mask (Sec. 3.2): <O, V> / |O|_1 =
// SumC(O . V) / SumC(O), the inverse by Goldschmidt's iteration on x = SumC(O) / N
// (y = 1 - x, a = 1 + y, b = y^2, then a <- a (1 + b), b <- b^2), the 1/N folded into
// the numerator; slot 0 of each query, zero if no element has rank k.
rk_ct* circuit_order_value_all(rk_ctx* c, const rk_ct* in, uint32_t k) {
    check_square(c, in, order_value_all_depth(c, in, k), "order value (all ties)");
    const double Nd = (double)in->N;
    Ev E{c};
    H O(circuit_order_stat(c, in, k, RK_TIES_ALL));
    H V(ct_clone_meta(in, in->level));
    ev_copy(c, in, V.p);
    H num = sum_cols(E, E.mul(O, E.level_down(V, O->level)), RK_MASK_COL0);
    H den = sum_cols(E, E.copy(O), RK_MASK_COL0);
    H x = E.mul_scalar(den, 1.0 / Nd);
    H y = E.add_const(E.neg(x), 1.0);
    H a = E.add_const(y, 1.0);
    H b = E.mul(y, y);
    a = E.level_down(a, b->level);
    for (int i = goldschmidt_iterations(in->N); i > 0; i--) {
        H a2 = E.mul(a, E.add_const(b, 1.0));
        b = E.mul(b, b);
        a = std::move(a2);
    }
    H numN = E.mul_scalar(num, 1.0 / Nd);
    const int lo = std::min(numN->level, a->level);
    return E.mul(E.level_down(numN, lo), E.level_down(a, lo)).release();
}

// Median (Alg. 4's particular case): the (N+1)/2-th statistic for odd N, else the mean
// of the N/2-th and (N/2+1)-th, as SumC((O_a + O_b) . V/2) on one shared rank; the two
// indicators run as one stack.
rk_ct* circuit_median(rk_ctx* c, const rk_ct* in) {
    check_square(c, in, order_value_depth(c, in), "median");
    const uint32_t N = in->N;
    const double Nd = (double)N;
    Ev E{c};
    H V(ct_clone_meta(in, in->level));
    ev_copy(c, in, V.p);
    H C = comparison_matrix(E, V, (int)c->prm.d_g, (int)c->prm.d_f);
    H R = sum_rows(E, tie_fold(E, C, RK_MASK_TIE), RK_MASK_ROW0S);
    const auto& co = indicator_coeffs(c, N);
    if (N % 2) {
        H O = cheb_ps(E, E.add_const(R, -(double)((N + 1) / 2) / Nd), co);
        return sum_cols(E, E.mul(O, E.level_down(V, O->level)), RK_MASK_COL0).release();
    }
    H ta = E.add_const(R, -(double)(N / 2) / Nd);
    H tb = E.add_const(R, -(double)(N / 2 + 1) / Nd);
    std::vector<rk_ct*> tp = {ta.p, tb.p};
    H O2 = cheb_ps(E, stack_of(c, tp), co);
    const int B = in->B;
    H M = E.add(range(O2, 0, B), range(O2, 1, B));
    H Vh = E.mul_scalar(V, 0.5);
    return sum_cols(E, E.mul(M, E.level_down(Vh, M->level)), RK_MASK_COL0).release();
}

int sort_depth(rk_ctx* c, const rk_ct* in) {
    const int dc = cmp_depth(c);
    return 1 + dc + 2 + 1 + cheb_depth((int)indicator_coeffs(c, in->N).size()) + 1 + 1;
}

// Alg. 5, column form (Sec. 3.3): C' = Cmp(V_C, V_R), tie fold ('tiec'), SumC / N, ReplC,
// minus (j+1)/N, Ind_0 gives M_ij = [r_i = j+1], SumR(M . V_C) is the sorted row.
rk_ct* circuit_sort(rk_ctx* c, const rk_ct* in, uint32_t flags) {
    (void)flags;
    check_square(c, in, sort_depth(c, in), "sort");
    Ev E{c};
    H V(ct_clone_meta(in, in->level));
    ev_copy(c, in, V.p);
    auto rc = row_col_forms(E, V);
    H Cc = cmp(E, E.sub(rc.second, rc.first), (int)c->prm.d_g, (int)c->prm.d_f);
    H S = sum_cols(E, tie_fold(E, Cc, RK_MASK_TIEC), RK_MASK_COL0S);
    H D = E.add_mask(repl_c(E, std::move(S)), RK_MASK_SORTIDX);
    H M = cheb_ps(E, D, indicator_coeffs(c, in->N));
    H Pm = E.mul(M, E.level_down(rc.second, M->level));
    return sum_r(E, std::move(Pm)).release();
}

// Stack of handles (copied) from a list of single ciphertexts or views.
static H stack_of(rk_ctx* c, const std::vector<rk_ct*>& xs) {
    std::vector<const rk_ct*> p(xs.begin(), xs.end());
    return H(ct_stack(c, p.data(), (int)p.size()));
}

static int stack_chunk(const rk_ctx* c, int level);

// f on the whole stack, in chunks of members that fit the stacking budget (members are
// independent, so the results are the same), or, when the context runs blocked
// circuits one ciphertext at a time (the plain per-query form), on each member with
// its own launches.
template <class F>
static H each(rk_ctx* c, Ev& E, H x, F f) {
    const int chunk = c->stack_blocks ? stack_chunk(c, x->level) : 1;
    if (x->B <= chunk) return f(std::move(x));
    std::vector<H> parts;
    std::vector<rk_ct*> ps;
    for (int b0 = 0; b0 < x->B; b0 += chunk) {
        const int g = std::min(chunk, x->B - b0);
        parts.push_back(f(E.copy(H(ct_view_range(x.p, b0, g)))));
        ps.push_back(parts.back().p);
    }
    return stack_of(c, ps);
}

// Members [i Bq, (i+1) Bq) of a stack built from L inputs of Bq members each.
static H range(const H& st, int i, int Bq) { return H(ct_view_range(st.p, i * Bq, Bq)); }

// outs[i] = a copy of members [i Bq, (i+1) Bq) (block i of every query)
static void split_blocks(rk_ctx* c, const H& st, int L, rk_ct** outs) {
    const int Bq = st->B / L;
    std::vector<rk_ct*> res(L, nullptr);
    try {
        for (int i = 0; i < L; i++) {
            H v = range(st, i, Bq);
            const rk_ct* one[1] = {v.p};
            res[i] = ct_stack(c, one, 1);
        }
    } catch (...) {
        for (auto* p : res) ct_free(p);
        throw;
    }
    for (int i = 0; i < L; i++) outs[i] = res[i];
}

static void check_blocks(rk_ctx* c, const rk_ct* const* blocks, int L, int need, const char* what) {
    RK_REQUIRE(L >= 1, RK_EINVAL, "no blocks");
    const rk_ct* b0 = blocks[0];
    for (int i = 0; i < L; i++)
        RK_REQUIRE(blocks[i]->B == b0->B && blocks[i]->level == b0->level && blocks[i]->N == b0->N &&
                       blocks[i]->Q == b0->Q && blocks[i]->n_real == b0->N,
                   RK_EINVAL, "blocks must be unpadded ciphertexts (or stacks of one size) of one level and length");
    check_square(c, b0, need, what);
}

// Tiles of Q B^2 slots a ciphertext of blocks shaped like `like` holds, when block-pair
// work may be packed into them: stacking on, packing on, at least two tiles, and the
// packing rotations' keys (left by +-T 2^s, 2^s below the tile count) present; else 1.
static int pair_tiles(const rk_ctx* c, const rk_ct* like) {
    if (!c->pair_packing || !c->stack_blocks) return 1;
    const size_t T = (size_t)like->Q * like->N * like->N;
    const size_t tiles = (size_t)c->n / 2 / T;
    if (tiles < 2) return 1;
    for (size_t s = 1; s < tiles; s <<= 1)
        for (int64_t r : {-(int64_t)(T * s), (int64_t)(T * s)})
            if (!c->gal.count(galois_left(c, (int)r))) return 1;
    return (int)tiles;
}

// f on each of the m members (Bq ciphertexts each) of the stack X, the members packed
// `per` to a ciphertext: member k of a group moves to tile k (slots k T + [0, T)) by a
// tree of stacked rotations (step s: x_i += x_(i+s) >> s T for every i whose place in
// its group is a multiple of 2s), f runs once on the stack of groups, and the results
// come back by the mirrored tree (entry j + s = entry j << s T).  f must act slot by
// slot and the members must be zero outside their first tile.  per = 1: f on X.
template <class F>
static H packed_apply(rk_ctx* c, Ev& E, H X, int m, int Bq, int T, int per, F f) {
    if (per <= 1) return f(std::move(X));
    std::vector<H> xs;
    for (int i = 0; i < m; i++) xs.push_back(E.copy(range(X, i, Bq)));
    X = H();
    for (int s = 1; s < per; s <<= 1) {
        std::vector<int> lo, hi;
        for (int i = 0; i < m; i++) {
            const int g = i % per;
            if (g % (2 * s) == 0 && g + s < per && i + s < m) {
                lo.push_back(i);
                hi.push_back(i + s);
            }
        }
        if (lo.empty()) continue;
        std::vector<rk_ct*> hp;
        for (int h : hi) hp.push_back(xs[h].p);
        H R = E.rot(stack_of(c, hp), -T * s);
        for (size_t p = 0; p < lo.size(); p++) xs[lo[p]] = E.add(xs[lo[p]], range(R, (int)p, Bq));
    }
    const int G = (m + per - 1) / per;
    std::vector<rk_ct*> gp;
    for (int g = 0; g < G; g++) gp.push_back(xs[g * per].p);
    H P = stack_of(c, gp);
    xs.clear();
    H Y = f(std::move(P));
    std::vector<H> parts(m);
    for (int g = 0; g < G; g++) parts[g * per] = E.copy(range(Y, g, Bq));
    for (int s = 1; s < per; s <<= 1) {
        std::vector<std::pair<int, int>> src;
        for (int g = 0; g < G; g++) {
            const int cnt = std::min(per, m - g * per);
            for (int j = 0; j < s && j + s < cnt; j++) src.push_back({g * per + j, g * per + j + s});
        }
        if (src.empty()) continue;
        std::vector<rk_ct*> sp;
        for (auto& pr : src) sp.push_back(parts[pr.first].p);
        H R = E.rot(stack_of(c, sp), T * s);
        for (size_t p = 0; p < src.size(); p++) parts[src[p].second] = E.copy(range(R, (int)p, Bq));
    }
    std::vector<rk_ct*> pp;
    for (auto& h : parts) pp.push_back(h.p);
    return stack_of(c, pp);
}

// Alg. 7 in two parts, so that the block comparisons (the parallel loop over block
// pairs of Sec. 5) can be spread over several devices and their partial sums exchanged.
// Part one: the comparisons C_{i,j} = Cmp(ReplR(V_i), ReplC(TransR(V_j))) of the listed
// pairs (j >= i), and per block the partial sums A_i = sum of the listed C_{i,j} and
// Bs_i = sum of the listed C_{j,i} with j < i (a zero ciphertext where no listed pair
// contributes), all at the comparison's output level.  The L blocks (one ciphertext
// each, same shape; each may be a stack of Bq members, block i of Bq queries) run as one
// stack through ReplR/TransR/ReplC, the listed comparisons as one stack through Cmp.
// Stack members of a step at `level` that fit the context's stacking budget: a member
// holds the key-switching scratch of one ciphertext and about a dozen live ciphertexts.
static int stack_chunk(const rk_ctx* c, int level) {
    const size_t l1 = (size_t)level + 1, QP = l1 + c->alpha;
    const size_t words = (l1 + (size_t)c->beta(level) * QP + 2 * QP + 7 * l1) + 24 * l1;
    return (int)std::max<size_t>(1, c->stack_budget_bytes / (words * c->n * 8));
}

// ReplR and ReplC(TransR) forms of L blocks (stacks of Bq each) as two stacks of L Bq,
// evaluated in chunks of blocks that fit the stacking budget (the same values as one
// stack: members are independent).
static std::pair<H, H> blocked_forms(rk_ctx* c, Ev& E, const rk_ct* const* blocks, int L) {
    const int Bq = blocks[0]->B;
    const int fc = std::max(1, stack_chunk(c, blocks[0]->level) / Bq);
    if (c->stack_blocks && fc >= L) {
        H V(ct_stack(c, blocks, L));
        return row_col_forms(E, V);
    }
    std::vector<H> fr, fcol;
    std::vector<rk_ct*> pr, pc;
    if (!c->stack_blocks) {   // the plain per-query form: every member on its own
        H V(ct_stack(c, blocks, L));
        for (int b = 0; b < V->B; b++) {
            auto f = row_col_forms(E, E.copy(H(ct_view(V.p, b))));
            fr.push_back(std::move(f.first));
            fcol.push_back(std::move(f.second));
        }
    } else {
        for (int b0 = 0; b0 < L; b0 += fc) {
            H V(ct_stack(c, blocks + b0, std::min(fc, L - b0)));
            auto f = row_col_forms(E, V);
            fr.push_back(std::move(f.first));
            fcol.push_back(std::move(f.second));
        }
    }
    for (auto& h : fr) pr.push_back(h.p);
    for (auto& h : fcol) pc.push_back(h.p);
    return std::make_pair(stack_of(c, pr), stack_of(c, pc));
}

void circuit_rank_blocked_partial(rk_ctx* c, const rk_ct* const* blocks, int L, const std::vector<std::pair<int, int>>& pairs,
                                  rk_ct** A_out, rk_ct** B_out) {
    const int need = 3 + cmp_depth(c);
    check_blocks(c, blocks, L, need, "blocked rank");
    for (auto& pr : pairs)
        RK_REQUIRE(pr.first >= 0 && pr.first <= pr.second && pr.second < L, RK_EINVAL, "block pair out of range");
    const int Bq = blocks[0]->B;
    Ev E{c};
    std::pair<H, H> rc = blocked_forms(c, E, blocks, L);   // stacks of L Bq
    const int lvl = rc.second->level - cmp_depth(c);
    std::vector<H> A(L), Bs(L);
    const int per = pair_tiles(c, blocks[0]);
    const int T = (int)(blocks[0]->Q * blocks[0]->N * blocks[0]->N);
    // the listed pairs in chunks that fit the stacking budget (whole packing groups)
    const size_t chunk = (size_t)std::max(1, stack_chunk(c, rc.second->level) / Bq) * per;
    for (size_t p0 = 0; p0 < pairs.size(); p0 += chunk) {
        const size_t p1 = std::min(pairs.size(), p0 + chunk);
        std::vector<H> vr_views, vc_views;
        std::vector<rk_ct*> vr, vc;
        for (size_t p = p0; p < p1; p++) {
            vr_views.push_back(range(rc.first, pairs[p].first, Bq));
            vc_views.push_back(range(rc.second, pairs[p].second, Bq));
            vr.push_back(vr_views.back().p);
            vc.push_back(vc_views.back().p);
        }
        H Cst = per > 1 ? packed_apply(c, E, E.sub(stack_of(c, vr), stack_of(c, vc)), (int)(p1 - p0), Bq, T, per,
                                       [&](H x) { return cmp(E, std::move(x), (int)c->prm.d_g, (int)c->prm.d_f); })
                        : each(c, E, E.sub(stack_of(c, vr), stack_of(c, vc)),
                               [&](H x) { return cmp(E, std::move(x), (int)c->prm.d_g, (int)c->prm.d_f); });
        for (size_t p = p0; p < p1; p++) {
            const int i = pairs[p].first, j = pairs[p].second;
            H Cij = range(Cst, (int)(p - p0), Bq);
            A[i] = A[i].p ? E.add(A[i], Cij) : E.copy(Cij);
            if (j > i) Bs[j] = Bs[j].p ? E.add(Bs[j], Cij) : E.copy(Cij);
        }
    }
    for (int i = 0; i < L; i++)
        for (H* h : {&A[i], &Bs[i]})
            if (!h->p) {   // no listed pair: an encryption of zero with no noise
                *h = H(ct_alloc_like(rc.second.p, lvl, Bq));
                RK_CUDA(cudaMemsetAsync((*h)->data, 0, (size_t)Bq * c->ct_words() * 8, c->stream));
                (*h)->level = lvl;
            }
    for (int i = 0; i < L; i++) {
        A_out[i] = A[i].release();
        B_out[i] = Bs[i].release();
    }
}

// Part two, given every pair's contribution summed over the parts:
// R_i = TransC(SumC(i - Bs_i)) + SumR(A_i) + 1/2 (Eq. 3: B_i = sum_{j<i} (1 - C_{j,i})).
void circuit_rank_blocked_finish(rk_ctx* c, const rk_ct* const* A_in, const rk_ct* const* B_in, int L, rk_ct** outs) {
    RK_REQUIRE(L >= 1, RK_EINVAL, "no blocks");
    const rk_ct* a0 = A_in[0];
    for (int i = 0; i < L; i++)
        RK_REQUIRE(A_in[i]->level == a0->level && B_in[i]->level == a0->level && A_in[i]->B == a0->B &&
                       B_in[i]->B == a0->B && A_in[i]->N == a0->N && B_in[i]->N == a0->N && A_in[i]->Q == a0->Q &&
                       B_in[i]->Q == a0->Q,
                   RK_EINVAL, "partial sums must share level, stack size and shape");
    RK_REQUIRE(a0->level >= 2, RK_EDEPTH, "blocked rank: the partial sums need two levels");
    const int Bq = a0->B;
    Ev E{c};
    std::vector<H> Bm;
    for (int i = 1; i < L; i++) Bm.push_back(E.add_const(E.neg(H(ct_view_range(B_in[i], 0, Bq))), (double)i));
    H S = each(c, E, H(ct_stack(c, A_in, L)), [&](H x) { return sum_r(E, std::move(x)); });   // stack of L Bq
    H T;
    if (L > 1) {
        std::vector<rk_ct*> bp;
        for (auto& b : Bm) bp.push_back(b.p);
        T = each(c, E, stack_of(c, bp), [&](H x) { return trans_c(E, sum_cols(E, std::move(x), RK_MASK_COL0)); });
    }
    std::vector<H> R;
    std::vector<rk_ct*> rp;
    for (int i = 0; i < L; i++) {
        H si = range(S, i, Bq);
        H r;
        if (i > 0) {
            H ti = range(T, i - 1, Bq);
            r = E.add(E.level_down(si, ti->level), ti);
        } else {
            r = E.level_down(si, si->level - 1);
        }
        R.push_back(E.add_const(r, 0.5));
        rp.push_back(R.back().p);
    }
    split_blocks(c, stack_of(c, rp), L, outs);
}

// Alg. 7 on one device: every pair (j >= i), then the assembly.
void circuit_rank_blocked(rk_ctx* c, const rk_ct* const* blocks, int L, rk_ct** outs) {
    std::vector<std::pair<int, int>> pairs;
    for (int i = 0; i < L; i++)
        for (int j = i; j < L; j++) pairs.push_back({i, j});
    std::vector<rk_ct*> A(L, nullptr), Bs(L, nullptr);
    try {
        circuit_rank_blocked_partial(c, blocks, L, pairs, A.data(), Bs.data());
        std::vector<const rk_ct*> a(A.begin(), A.end()), b(Bs.begin(), Bs.end());
        circuit_rank_blocked_finish(c, a.data(), b.data(), L, outs);
    } catch (...) {
        for (auto* p : A) ct_free(p);
        for (auto* p : Bs) ct_free(p);
        throw;
    }
    for (auto* p : A) ct_free(p);
    for (auto* p : Bs) ct_free(p);
}

// 2 C^2 - C: 1 where the row-form value exceeds the column-form value, 0 at ties
// (Cmp_G of Sec. 3.2).
static H cmp_strict(Ev& E, const H& C) {
    H C2 = E.mul(C, C);
    return E.sub(E.add(C2, C2), E.level_down(C, C2->level));
}

// ReplR (Alg. 10): X <- X + (X >> N 2^i)
static H repl_r(Ev& E, H x) {
    const int N = (int)x->N, k = log2_exact(x->N);
    return chain(E, std::move(x), repl_r_amounts(N, k));
}

static int blocked_rank_tc_depth(const rk_ctx* c) { return 1 + cmp_depth(c) + 3; }

// Tie-corrected ranks of a multi-ciphertext vector (Alg. 7 with Alg. 6 across blocks).
// The rank of element b of block i counts the smaller values and the equal values at
// an earlier global position (earlier block, or same block and position <= b):
//   pair j = i:  SumR(C_ii + E_ii (delta - 1/2))   (the folded single-block offset)
//   pair j > i:  SumR(G_ij),  G = 2C^2 - C        (strictly smaller values of block j)
//   pair j < i:  TransC(SumC(1 - G_ji))           (values of block j not larger, Eq. 3)
// The diagonal and the upper pairs each run as one stack.  `scaled` divides every rank
// by D = L B in the row masks.  Returns the stack of the L rank blocks and the stack
// of the blocks' ReplR forms.
static std::pair<H, H> blocked_ranks_tc(rk_ctx* c, const rk_ct* const* blocks, int L, bool scaled) {
    Ev E{c};
    const int Bsz = (int)blocks[0]->N, Bq = blocks[0]->B, dg = (int)c->prm.d_g, df = (int)c->prm.d_f;
    const uint32_t Dn = scaled ? (uint32_t)(L * Bsz) : 0u;
    const uint32_t rmask = scaled ? RK_MASK_ROW0S : RK_MASK_ROW0;
    auto rc = blocked_forms(c, E, blocks, L);   // stacks of L Bq
    std::vector<H> views;
    std::vector<rk_ct*> dr, dcol;
    std::vector<std::pair<int, int>> up;
    for (int i = 0; i < L; i++) {
        views.push_back(range(rc.first, i, Bq));
        dr.push_back(views.back().p);
        views.push_back(range(rc.second, i, Bq));
        dcol.push_back(views.back().p);
    }
    for (int i = 0; i < L; i++)
        for (int j = i + 1; j < L; j++) up.push_back({i, j});
    const int per = pair_tiles(c, blocks[0]);
    const int tile = (int)(blocks[0]->Q * Bsz * Bsz);
    // members in chunks that fit the stacking budget (whole packing groups)
    const size_t chunk = (size_t)std::max(1, stack_chunk(c, rc.second->level) / Bq) * per;
    std::vector<H> Fparts;
    std::vector<rk_ct*> fp;
    for (size_t i0 = 0; i0 < (size_t)L; i0 += chunk) {
        const size_t i1 = std::min((size_t)L, i0 + chunk);
        std::vector<rk_ct*> r(dr.begin() + i0, dr.begin() + i1), cl(dcol.begin() + i0, dcol.begin() + i1);
        Fparts.push_back(tie_fold(E, packed_apply(c, E, E.sub(stack_of(c, r), stack_of(c, cl)), (int)(i1 - i0), Bq, tile, per,
                                                  [&](H x) { return cmp(E, std::move(x), dg, df); }),
                                  RK_MASK_TIE));
        fp.push_back(Fparts.back().p);
    }
    H F = Fparts.size() == 1 ? std::move(Fparts[0]) : stack_of(c, fp);
    Fparts.clear();
    // A_i = F_i + sum_{j > i} G_ij (at F's level), Bs_i = sum_{j < i} G_ji, in pair order
    std::vector<H> A(L), Bsum(L);
    for (int i = 0; i < L; i++) A[i] = E.copy(range(F, i, Bq));
    for (size_t p0 = 0; p0 < up.size(); p0 += chunk) {
        const size_t p1 = std::min(up.size(), p0 + chunk);
        std::vector<rk_ct*> r, cl;
        for (size_t p = p0; p < p1; p++) {
            r.push_back(dr[up[p].first]);
            cl.push_back(dcol[up[p].second]);
        }
        H G = packed_apply(c, E, E.sub(stack_of(c, r), stack_of(c, cl)), (int)(p1 - p0), Bq, tile, per,
                           [&](H x) { return cmp_strict(E, cmp(E, std::move(x), dg, df)); });
        H Gd = E.level_down(G, F->level);
        for (size_t p = p0; p < p1; p++) {
            const int i = up[p].first, j = up[p].second;
            A[i] = E.add(A[i], range(Gd, (int)(p - p0), Bq));
            H gji = range(G, (int)(p - p0), Bq);
            Bsum[j] = Bsum[j].p ? E.add(Bsum[j], gji) : E.copy(gji);
        }
    }
    std::vector<H> Bm;
    for (int i = 1; i < L; i++) Bm.push_back(E.add_const(E.neg(Bsum[i]), (double)i));
    std::vector<rk_ct*> ap;
    for (auto& a : A) ap.push_back(a.p);
    const int kB = log2_exact((uint32_t)Bsz);
    H S = each(c, E, stack_of(c, ap), [&](H x) {
        return E.mul_mask_d(chain(E, std::move(x), pow2_amounts(Bsz, kB, 1)), rmask, Dn);
    });
    A.clear();
    if (L == 1) return std::make_pair(std::move(S), std::move(rc.first));
    std::vector<rk_ct*> bp;
    for (auto& b : Bm) bp.push_back(b.p);
    H T = each(c, E, stack_of(c, bp), [&](H x) {   // stack of (L - 1) Bq
        return E.mul_mask_d(chain(E, sum_cols(E, std::move(x), RK_MASK_COL0), negated(trans_r_amounts(Bsz, kB))), rmask, Dn);
    });
    Bm.clear();
    std::vector<H> R;
    std::vector<rk_ct*> rp;
    for (int i = 0; i < L; i++) {
        H si = range(S, i, Bq);
        if (i == 0) {
            R.push_back(E.copy(si));
        } else {
            H ti = range(T, i - 1, Bq);
            R.push_back(E.add(si, E.level_down(ti, si->level)));
        }
        rp.push_back(R.back().p);
    }
    return std::make_pair(stack_of(c, rp), std::move(rc.first));
}

void circuit_rank_blocked_tc(rk_ctx* c, const rk_ct* const* blocks, int L, rk_ct** outs) {
    check_blocks(c, blocks, L, blocked_rank_tc_depth(c), "blocked rank");
    auto rr = blocked_ranks_tc(c, blocks, L, false);
    split_blocks(c, rr.first, L, outs);
}

// Alg. 4 on the tie-corrected blocked ranks: O_i = Ind_k(R_i), the indicator the
// sinc^2 window for the whole length D = L B; the L blocks run as one stack.
void circuit_order_stat_blocked(rk_ctx* c, const rk_ct* const* blocks, int L, uint32_t k, rk_ct** outs) {
    RK_REQUIRE(L >= 1, RK_EINVAL, "no blocks");
    const uint32_t D = (uint32_t)L * blocks[0]->N;
    RK_REQUIRE(k >= 1 && k <= D, RK_EINVAL, "k must be in [1, L B]");
    const auto& co = indicator_coeffs(c, D);
    check_blocks(c, blocks, L, blocked_rank_tc_depth(c) + cheb_depth((int)co.size()), "blocked order statistic");
    auto rr = blocked_ranks_tc(c, blocks, L, true);
    Ev E{c};
    const int Bq = blocks[0]->B, per = pair_tiles(c, blocks[0]);
    const int T = (int)(blocks[0]->Q * blocks[0]->N * blocks[0]->N);
    // the L indicators in chunks of whole packing groups that fit the indicator budget
    const size_t ct_bytes = (size_t)2 * (rr.first->level + 1) * c->n * 8 * Bq;
    const size_t live = (size_t)baby_steps((int)co.size()) + 2 * (size_t)cheb_depth((int)co.size()) + 8;
    const int chunk = (int)std::max<size_t>(1, c->ind_stack_bytes / (live * ct_bytes)) * per;
    std::vector<H> parts;
    std::vector<rk_ct*> pp;
    for (int i0 = 0; i0 < L; i0 += chunk) {
        const int i1 = std::min(L, i0 + chunk);
        parts.push_back(packed_apply(c, E, H(ct_view_range(rr.first.p, i0 * Bq, (i1 - i0) * Bq)), i1 - i0, Bq, T, per,
                                     [&](H x) { return cheb_ps(E, E.add_const(x, -(double)k / D), co); }));
        pp.push_back(parts.back().p);
    }
    H O = parts.size() == 1 ? std::move(parts[0]) : stack_of(c, pp);
    split_blocks(c, O, L, outs);
}

// Alg. 8 on the tie-corrected blocked ranks:
//   S_i = TransC(SumC(sum_j Ind_0(ReplR(R_j) - offset_i) . ReplR(V_j)))
// offset_i holds B i + a + 1 in row a: the mask RK_MASK_ROWIDX plus the constant
// -B i / D (ranks and offsets divided by D = L B).  The L^2 indicators run as stacks of
// at most `chunk` pairs so that the Paterson-Stockmeyer working set stays bounded.
void circuit_sort_blocked(rk_ctx* c, const rk_ct* const* blocks, int L, rk_ct** outs) {
    RK_REQUIRE(L >= 1, RK_EINVAL, "no blocks");
    const int Bsz = (int)blocks[0]->N, Bq = blocks[0]->B;
    const uint32_t D = (uint32_t)(L * Bsz);
    const auto& co = indicator_coeffs(c, D);
    check_blocks(c, blocks, L, blocked_rank_tc_depth(c) + cheb_depth((int)co.size()) + 3, "blocked sort");
    auto rr = blocked_ranks_tc(c, blocks, L, true);
    Ev E{c};
    H RR = each(c, E, std::move(rr.first), [&](H x) {   // stack of L Bq
        return E.add_mask_d(repl_r(E, std::move(x)), RK_MASK_ROWIDX, D);
    });
    const size_t ct_bytes = (size_t)2 * (RR->level + 1) * c->n * 8 * Bq;
    const size_t live = (size_t)baby_steps((int)co.size()) + 2 * (size_t)cheb_depth((int)co.size()) + 8;
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)L * L, c->ind_stack_bytes / (live * ct_bytes)));
    std::vector<H> acc(L);
    const int per = pair_tiles(c, blocks[0]);
    if (per > 1) {
        // per output block i, its L indicators packed `per` to a ciphertext: the RR_j
        // (zero outside their tile) packed, the constant -B i / D added to every slot
        const int T = (int)(blocks[0]->Q * Bsz * Bsz);
        const int jc = std::max(1, chunk) * per;   // whole packing groups a chunk
        for (int i = 0; i < L; i++) {
            for (int j0 = 0; j0 < L; j0 += jc) {
                const int j1 = std::min(L, j0 + jc);
                H M = packed_apply(c, E, E.copy(H(ct_view_range(RR.p, j0 * Bq, (j1 - j0) * Bq))), j1 - j0, Bq, T, per,
                                   [&](H x) { return cheb_ps(E, E.add_const(x, -(double)Bsz * i / D), co); });
                std::vector<H> vr;
                std::vector<rk_ct*> vp;
                for (int j = j0; j < j1; j++) {
                    vr.push_back(E.level_down(range(rr.second, j, Bq), M->level));
                    vp.push_back(vr.back().p);
                }
                H P = E.mul(M, stack_of(c, vp));
                for (int j = j0; j < j1; j++) {
                    H pm = range(P, j - j0, Bq);
                    acc[i] = acc[i].p ? E.add(acc[i], pm) : E.copy(pm);
                }
            }
        }
    }
    std::vector<std::pair<int, int>> pairs;
    for (int i = 0; i < L && per <= 1; i++)
        for (int j = 0; j < L; j++) pairs.push_back({i, j});
    for (size_t p0 = 0; p0 < pairs.size(); p0 += chunk) {
        const size_t p1 = std::min(pairs.size(), p0 + chunk);
        std::vector<H> in, vr;
        std::vector<rk_ct*> ip;
        for (size_t p = p0; p < p1; p++) {
            in.push_back(E.add_const(range(RR, pairs[p].second, Bq), -(double)Bsz * pairs[p].first / D));
            ip.push_back(in.back().p);
        }
        H M = cheb_ps(E, stack_of(c, ip), co);
        in.clear();
        std::vector<rk_ct*> vp;
        for (size_t p = p0; p < p1; p++) {
            vr.push_back(E.level_down(range(rr.second, pairs[p].second, Bq), M->level));
            vp.push_back(vr.back().p);
        }
        H P = E.mul(M, stack_of(c, vp));
        for (size_t p = p0; p < p1; p++) {
            H pm = range(P, (int)(p - p0), Bq);
            const int i = pairs[p].first;
            acc[i] = acc[i].p ? E.add(acc[i], pm) : E.copy(pm);
        }
    }
    std::vector<rk_ct*> ap;
    for (auto& a : acc) ap.push_back(a.p);
    H S = trans_c(E, sum_cols(E, stack_of(c, ap), RK_MASK_COL0));
    split_blocks(c, S, L, outs);
}

rk_ct* circuit_compare_matrix(rk_ctx* c, const rk_ct* in) {
    RK_REQUIRE(in->layout == RK_LAYOUT_ROW, RK_EINVAL, "compare_matrix expects a row vector");
    RK_REQUIRE((size_t)in->Q * in->N * in->N <= (size_t)c->n / 2, RK_EINVAL, "N^2 exceeds the slots");
    const int need = 1 + cmp_depth(c);
    RK_REQUIRE(in->level >= need, RK_EDEPTH, "comparison needs " + std::to_string(need) + " levels");
    RK_REQUIRE(cmp_ok(c), RK_EINVAL, "comparator needs at least one stage");
    Ev E{c};
    H V(ct_clone_meta(in, in->level));
    ev_copy(c, in, V.p);
    return comparison_matrix(E, V, (int)c->prm.d_g, (int)c->prm.d_f).release();
}

// Rotation amounts the circuits use for a vector of length N (Sec. 3.1 and App. A):
// every chain's steps (ReplR, SumR, ReplC, SumC, TransR, TransC) and the sums of the
// step pairs the chains take two at a time (steps 2j and 2j + 1).
void circuit_rotations(uint32_t N, std::vector<int>& out) {
    const int k = log2_exact(N);
    const int n = (int)N;
    const std::vector<std::vector<int>> chains = {repl_r_amounts(n, k), pow2_amounts(n, k, 1), pow2_amounts(1, k, -1),
                                                  pow2_amounts(1, k, 1), trans_r_amounts(n, k), negated(trans_r_amounts(n, k))};
    for (const auto& ch : chains) {
        for (int a : ch) out.push_back(a);
        for (size_t i = 0; i + 1 < ch.size(); i += 2) out.push_back(ch[i] + ch[i + 1]);
    }
}
