// Homomorphic operations of RNS-CKKS on the device (Sec. 2.1: addition,
// multiplication, rotation), key generation and the client operations.
//
// Conventions (fixed by this library; the paper leaves them to the scheme):
//  * hybrid key switching with digits of `digit_size` limbs; ModUp is the fast
//    basis conversion of one digit without correction; for a rotation the
//    automorphism X -> X^g acts on the lifted digits (so that several rotations of
//    one ciphertext share one ModUp); ModDown converts the P part back with centred
//    terms (zero-mean error) and multiplies by P^-1;
//  * rescale lifts the dropped residue centred into (-q/2, q/2];
//  * a factor (scalar or plaintext) multiplied at level l is encoded at scale
//    Delta_{l-1} q_l / Delta_l and rounded half away from zero, so that after the
//    rescale the product sits at the canonical scale Delta_{l-1};
//  * a constant c is added as round(c Delta_l) to every evaluation of c0.
//
// A handle may hold a stack of B ciphertexts ([B][2][L+1][n]); every operation
// then runs on all of them with the same launches (same constants, same keys).
#include <cmath>
#include <complex>
#include <cstring>

#include "kernels.cuh"

namespace {

struct Scratch {
    u64 *coef, *ext, *u, *w, *d, *v, *misc;
    size_t misc_words;
};

// Regions sized for stacks of up to c->batch_cap ciphertexts at the top level.
Scratch scratch_layout(rk_ctx* c) {
    const size_t n = c->n, L1 = c->L + 1, QP = c->L + 1 + c->alpha, Bc = (size_t)c->batch_cap;
    const size_t w_coef = Bc * L1 * n, w_ext = Bc * (size_t)c->beta(c->L) * QP * n, w_u = Bc * 2 * QP * n,
                 w_w = Bc * 2 * L1 * n, w_d = Bc * 3 * L1 * n, w_v = Bc * 2 * L1 * n, w_misc = 4 * QP * n;
    u64* b = c->scratch(w_coef + w_ext + w_u + w_w + w_d + w_v + w_misc);
    Scratch S;
    S.coef = b;
    S.ext = S.coef + w_coef;
    S.u = S.ext + w_ext;
    S.w = S.u + w_u;
    S.d = S.w + w_w;
    S.v = S.d + w_d;
    S.misc = S.v + w_v;
    S.misc_words = w_misc;
    return S;
}

LimbSet ls_q(u64* base, size_t ps, int polys, int limbs) { return LimbSet{base, ps, polys, limbs, limbs, 0, 0}; }
LimbSet ls_one(u64* base, size_t ps, int polys, int prime) { return LimbSet{base, ps, polys, 1, 1, prime, 0}; }
LimbSet ls_all(u64* base, size_t ps, int polys, int np) { return LimbSet{base, ps, polys, np, np, 0, 0}; }

u64 shoup_companion(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

ScalarArg scalar_residues(const rk_ctx* c, int64_t K, int limbs) {
    ScalarArg a;
    memset(&a, 0, sizeof(a));
    for (int i = 0; i < limbs; i++) {
        const int64_t q = (int64_t)c->primes[i];
        int64_t r = K % q;
        if (r < 0) r += q;
        a.w[i] = (u64)r;
        a.wsh[i] = shoup_companion((u64)r, (u64)q);
    }
    return a;
}

// SplitMix64 counter stream for host-side sampling (keys, encryption noise).
struct HostRng {
    u64 seed, ctr = 0;
    explicit HostRng(u64 s) : seed(s) {}
    static u64 mix(u64 x) {
        x += 0x9E3779B97F4A7C15ull;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        return x ^ (x >> 31);
    }
    u64 next() { return mix(seed ^ mix(ctr++)); }
    double uniform01() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    int64_t ternary() { return (int64_t)(next() % 3) - 1; }
    int64_t gaussian(double sigma) {
        for (;;) {
            double u1 = uniform01(), u2 = uniform01();
            double g = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2) * sigma;
            if (std::fabs(g) <= 6.0 * sigma) return (int64_t)llround(g);
        }
    }
};

const double kSigma = 3.19;

void upload_i64_sync(rk_ctx* c, int64_t* dst, const int64_t* src, size_t count) {
    RK_CUDA(cudaMemcpyAsync(dst, src, count * 8, cudaMemcpyHostToDevice, c->stream));
    RK_CUDA(cudaStreamSynchronize(c->stream));
}

// copy limbs 0..l of `polys` polynomials between two buffers with poly stride ps
void copy_polys(rk_ctx* c, u64* dst, const u64* src, int polys, int l) {
    const size_t pitch = c->poly_stride() * 8, width = (size_t)(l + 1) * c->n * 8;
    RK_CUDA(cudaMemcpy2DAsync(dst, pitch, src, pitch, width, polys, cudaMemcpyDeviceToDevice, c->stream));
}

}  // namespace

void ensure_batch(rk_ctx* c, int B) {
    if (B > c->batch_cap) {
        c->batch_cap = B;
        scratch_layout(c);   // grows the allocation (synchronises once)
    }
}

// ---------------------------------------------------------------------------
// Ciphertext handles
// ---------------------------------------------------------------------------
rk_ct* ct_alloc(rk_ctx* c, int level, int B) {
    rk_ct* ct = new rk_ct();
    ct->ctx = c;
    ct->level = level;
    ct->B = B;
    cudaError_t e = rk_malloc_async((void**)&ct->data, (size_t)B * c->ct_words() * 8, c->stream);
    if (e != cudaSuccess) {
        delete ct;
        throw rk_error(RK_ENOMEM, std::string("ciphertext allocation: ") + cudaGetErrorString(e));
    }
    return ct;
}

void ct_free(rk_ct* ct) {
    if (!ct) return;
    if (ct->data && !ct->view) cudaFreeAsync(ct->data, ct->ctx->stream);
    delete ct;
}

rk_ct* ct_view(const rk_ct* stack, int b) { return ct_view_range(stack, b, 1); }

rk_ct* ct_view_range(const rk_ct* stack, int first, int count) {
    RK_REQUIRE(first >= 0 && count >= 1 && first + count <= stack->B, RK_EINVAL, "view range out of range");
    rk_ct* v = new rk_ct(*stack);
    v->data = stack->data + (size_t)first * stack->ctx->ct_words();
    v->B = count;
    v->view = true;
    return v;
}

static void copy_meta(rk_ct* out, const rk_ct* a) {
    out->N = a->N;
    out->n_real = a->n_real;
    out->Q = a->Q;
    out->layout = a->layout;
}

rk_ct* ct_clone_meta(const rk_ct* src, int level) {
    rk_ct* o = ct_alloc(src->ctx, level, src->B);
    copy_meta(o, src);
    return o;
}
rk_ct* ct_stack(rk_ctx* c, const rk_ct* const* in, int count) {
    RK_REQUIRE(count >= 1, RK_EINVAL, "stack of no ciphertexts");
    const rk_ct* a = in[0];
    int total = 0;
    for (int i = 0; i < count; i++) {
        RK_REQUIRE(in[i]->level == a->level && in[i]->N == a->N && in[i]->Q == a->Q && in[i]->n_real == a->n_real &&
                       in[i]->layout == a->layout,
                   RK_EINVAL, "stacked ciphertexts must share level and vector shape");
        total += in[i]->B;
    }
    rk_ct* o = ct_alloc(c, a->level, total);
    copy_meta(o, a);
    int at = 0;
    for (int i = 0; i < count; i++) {   // members of a stacked input keep their order
        copy_polys(c, o->data + (size_t)at * c->ct_words(), in[i]->data, 2 * in[i]->B, a->level);
        at += in[i]->B;
    }
    return o;
}

void ct_unstack(rk_ctx* c, const rk_ct* in, rk_ct** outs) {
    for (int i = 0; i < in->B; i++) {
        rk_ct* o = ct_alloc(c, in->level, 1);
        copy_meta(o, in);
        copy_polys(c, o->data, in->data + (size_t)i * c->ct_words(), 2, in->level);
        outs[i] = o;
    }
}

// ---------------------------------------------------------------------------
// Pointwise operations
// ---------------------------------------------------------------------------
void ev_copy(rk_ctx* c, const rk_ct* a, rk_ct* out) {
    RK_REQUIRE(out->B == a->B, RK_EINVAL, "copy: stack size mismatch");
    if (out != a) copy_polys(c, out->data, a->data, 2 * a->B, a->level);
    out->level = a->level;
    copy_meta(out, a);
}

void ev_add(rk_ctx* c, const rk_ct* a, const rk_ct* b, rk_ct* out) {
    RK_REQUIRE(a->level == b->level, RK_EINVAL, "add: level mismatch");
    RK_REQUIRE(a->B == b->B && out->B == a->B, RK_EINVAL, "add: stack size mismatch");
    launch_addsub(c->env, out->data, a->data, b->data, a->level + 1, c->poly_stride(), 0, c->stream, 2 * a->B);
    out->level = a->level;
    copy_meta(out, a);
}

void ev_sub(rk_ctx* c, const rk_ct* a, const rk_ct* b, rk_ct* out) {
    RK_REQUIRE(a->level == b->level, RK_EINVAL, "sub: level mismatch");
    RK_REQUIRE(a->B == b->B && out->B == a->B, RK_EINVAL, "sub: stack size mismatch");
    launch_addsub(c->env, out->data, a->data, b->data, a->level + 1, c->poly_stride(), 1, c->stream, 2 * a->B);
    out->level = a->level;
    copy_meta(out, a);
}

void ev_neg(rk_ctx* c, const rk_ct* a, rk_ct* out) {
    launch_addsub(c->env, out->data, a->data, a->data, a->level + 1, c->poly_stride(), 2, c->stream, 2 * a->B);
    out->level = a->level;
    copy_meta(out, a);
}

void ev_add_const(rk_ctx* c, const rk_ct* a, double v, rk_ct* out) {
    const int l = a->level;
    const int64_t K = round_half_away(v * c->scales[l]);
    launch_add_const(c->env, out->data, a->data, scalar_residues(c, K, l + 1), l + 1, c->poly_stride(), c->stream, 2 * a->B);
    out->level = l;
    copy_meta(out, a);
}

// Rescale of `a` (level l) into `out` (level l - 1): out_i = (K_i a_i - v_i) q_l^-1,
// i < l, where v is the centred lift of the last limb of `out` (which must hold
// K_l a_l) taken back to the evaluation domain.  K null means K = 1 (out may be a);
// otherwise it is the scalar product fused with its rescale.
static void rescale_into(rk_ctx* c, const rk_ct* a, const ScalarArg* K, rk_ct* out) {
    const int l = a->level;
    ensure_batch(c, a->B);
    Scratch S = scratch_layout(c);
    const size_t ps = c->poly_stride(), n = c->n;
    const int polys = 2 * a->B;
    u64* last = out->data + (size_t)l * n;
    launch_ntt_inverse(c->env, ls_one(last, ps, polys, l), c->stream);
    LimbSet v = ls_q(S.v, (size_t)l * n, polys, l);   // the lift happens in the first forward pass
    v.lift = last;
    v.lift_stride = ps;
    v.lift_mod = c->env.conv.rescale + (size_t)l * 3 * (c->L + 1) + 2 * (c->L + 1);
    v.lift_q = c->primes[l];
    launch_ntt_forward(c->env, v, c->stream);
    launch_rescale_combine(c->env, out->data, a->data, ps, S.v, l, K, c->stream, polys);
    out->level = l - 1;
    c->n_rescale++;
}

void ev_rescale_inplace(rk_ctx* c, rk_ct* a) {
    RK_REQUIRE(a->level >= 1, RK_EDEPTH, "rescale: no level left");
    rescale_into(c, a, nullptr, a);
}

static double factor_scale(const rk_ctx* c, int l) {
    return (c->scales[l - 1] * (double)c->primes[l]) / c->scales[l];
}

void ev_mul_scalar(rk_ctx* c, const rk_ct* a, double v, rk_ct* out) {
    const int l = a->level;
    RK_REQUIRE(l >= 1, RK_EDEPTH, "mul_scalar: no level left");
    RK_REQUIRE(out->B == a->B, RK_EINVAL, "mul_scalar: stack size mismatch");
    const int64_t K = round_half_away(v * factor_scale(c, l));
    const ScalarArg Kr = scalar_residues(c, K, l + 1);
    // the product's last limb only; the other limbs are scaled inside the rescale
    launch_mul_scalar(c->env, out->data, a->data, Kr, 1, c->poly_stride(), c->stream, 2 * a->B, l);
    copy_meta(out, a);
    out->level = l;
    rescale_into(c, a, &Kr, out);
}

void ev_level_down(rk_ctx* c, const rk_ct* a, int target, rk_ct* out) {
    RK_REQUIRE(target <= a->level && target >= 0, RK_EINVAL, "level_down: bad target");
    if (a->level == target) {
        ev_copy(c, a, out);
        return;
    }
    ev_mul_scalar(c, a, 1.0, out);
    while (out->level > target) ev_mul_scalar(c, out, 1.0, out);
}

const std::vector<double>& encoding_of(rk_ctx* c, uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real) {
    auto ekey = std::make_tuple(kind, N, Q, n_real);
    if (!c->encodings.count(ekey)) {
        std::vector<double> slots;
        mask_slot_values(kind, N, Q, n_real, (size_t)c->n / 2, slots);
        std::vector<double> u;
        encode_unscaled(c->log_n, slots.data(), slots.size(), u);
        c->encodings[ekey] = u;
    }
    return c->encodings[ekey];
}

// Residues of round(s u) over limbs 0..l in the evaluation domain (Montgomery form if mont).
static u64* plain_make(rk_ctx* c, const std::vector<double>& u, double s, int l, bool mont) {
    std::vector<int64_t> m(c->n);
    for (int k = 0; k < c->n; k++) m[k] = round_half_away(s * u[k]);
    Scratch S = scratch_layout(c);
    u64* buf = nullptr;
    RK_CUDA(rk_malloc((void**)&buf, (size_t)(l + 1) * c->n * 8));
    int64_t* tmp = (int64_t*)S.misc;
    upload_i64_sync(c, tmp, m.data(), c->n);
    launch_reduce_signed(c->env, tmp, ls_q(buf, 0, 1, l + 1), c->stream);
    launch_ntt_forward(c->env, ls_q(buf, 0, 1, l + 1), c->stream);
    if (mont) launch_to_mont(c->env, ls_q(buf, 0, 1, l + 1), c->stream);
    RK_CUDA(cudaStreamSynchronize(c->stream));
    return buf;
}

static const u64* plain_get(rk_ctx* c, uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real, int l) {
    auto key = std::make_tuple(kind, N, Q, n_real, l);
    auto it = c->plain_cache.find(key);
    if (it != c->plain_cache.end()) return it->second;
    u64* buf = plain_make(c, encoding_of(c, kind, N, Q, n_real), factor_scale(c, l), l, true);
    c->plain_cache[key] = buf;
    return buf;
}

// Mask plaintext encoded at the canonical scale Delta_l (normal form), for addition.
static const u64* plain_add_get(rk_ctx* c, uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real, int l) {
    auto key = std::make_tuple(kind, N, Q, n_real, l);
    auto it = c->plain_add_cache.find(key);
    if (it != c->plain_add_cache.end()) return it->second;
    u64* buf = plain_make(c, encoding_of(c, kind, N, Q, n_real), c->scales[l], l, false);
    c->plain_add_cache[key] = buf;
    return buf;
}

void ev_mul_plain(rk_ctx* c, const rk_ct* a, uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real, rk_ct* out) {
    const int l = a->level;
    RK_REQUIRE(l >= 1, RK_EDEPTH, "mul_plain: no level left");
    const u64* pt = plain_get(c, kind, N, Q, n_real, l);
    launch_mul_plain(c->env, out->data, a->data, pt, l + 1, c->poly_stride(), c->stream, 2 * a->B);
    out->level = l;
    copy_meta(out, a);
    ev_rescale_inplace(c, out);
}

void ev_add_plain(rk_ctx* c, const rk_ct* a, uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real, rk_ct* out) {
    const int l = a->level;
    const u64* pt = plain_add_get(c, kind, N, Q, n_real, l);
    const size_t cw = c->ct_words();
    for (int b = 0; b < a->B; b++)   // c0 + pt for every stacked ciphertext
        launch_addsub(c->env, out->data + b * cw, a->data + b * cw, pt, l + 1, 0, 0, c->stream, 1);
    if (out != a)
        for (int b = 0; b < a->B; b++) copy_polys(c, out->data + b * cw + c->poly_stride(), a->data + b * cw + c->poly_stride(), 1, l);
    out->level = l;
    copy_meta(out, a);
}

rk_ct* ct_alloc_like(const rk_ct* like, int level, int B) {
    rk_ct* o = ct_alloc(like->ctx, level, B);
    copy_meta(o, like);
    return o;
}

void ev_lincomb(rk_ctx* c, const std::vector<const rk_ct*>& xs, const std::vector<double>& cs, rk_ct* out, bool rescale) {
    RK_REQUIRE(!xs.empty() && xs.size() == cs.size(), RK_EINVAL, "lincomb: bad term lists");
    const int l = xs[0]->level;
    RK_REQUIRE(l >= 1, RK_EDEPTH, "lincomb: no level left");
    for (auto* x : xs) RK_REQUIRE(x->level == l && x->B == out->B, RK_EINVAL, "lincomb: level or stack mismatch");
    for (auto* x : xs) RK_REQUIRE(x != out, RK_EINVAL, "lincomb: output aliases an input");
    const double s = factor_scale(c, l);
    LincombArg arg;
    size_t done = 0;
    while (done < xs.size()) {
        const int terms = (int)std::min<size_t>(16, xs.size() - done);
        for (int i = 0; i < terms; i++) {
            arg.x[i] = xs[done + i]->data;
            const int64_t K = round_half_away(cs[done + i] * s);
            for (int t = 0; t <= l; t++) {
                const int64_t q = (int64_t)c->primes[t];
                int64_t r = K % q;
                if (r < 0) r += q;
                arg.KR[i][t] = h_mulmod((u64)r, c->h_pc[t].r_mod, (u64)q);
            }
        }
        launch_lincomb(c->env, out->data, arg, terms, done > 0, l + 1, c->poly_stride(), c->stream, 2 * out->B);
        done += terms;
    }
    out->level = l;
    copy_meta(out, xs[0]);
    if (rescale) ev_rescale_inplace(c, out);
}

// ---------------------------------------------------------------------------
// Key switching
// ---------------------------------------------------------------------------
// ModUp, first half: B polynomials d_b = d_eval + b * d_stride (evaluation domain,
// limbs 0..l) to the coefficient domain in S.coef [B][l+1][n].
static void ks_lift(rk_ctx* c, const u64* d_eval, size_t d_stride, int l, int B) {
    ensure_batch(c, B);
    Scratch S = scratch_layout(c);
    const size_t n = c->n;
    LimbSet s = ls_q(S.coef, (size_t)(l + 1) * n, B, l + 1);
    s.src = d_eval;   // the first pass reads the input, the transform lands in S.coef
    s.src_stride = d_stride;
    launch_ntt_inverse(c->env, s, c->stream);
}

// Staged ModUp, second half: every digit lifted to the ext scratch
// [B][beta][l+1+alpha][n] and taken to the evaluation domain in place.
static void ks_lift_ext(rk_ctx* c, const u64* d_eval, size_t d_stride, int l, int B) {
    Scratch S = scratch_layout(c);
    const size_t n = c->n;
    const int QP = l + 1 + c->alpha;
    LimbSet ext{S.ext, (size_t)QP * n, B * c->beta(l), QP, l + 1, 0, c->L + 1};
    ext.skip_ds = c->dsize;   // each digit's own limbs are already in the evaluation domain
    ext.skip_beta = c->beta(l);
    if (c->modup_col) {   // conversion fused into the column pass, then the row pass
        launch_modup_col(c->env, S.coef, S.ext, (size_t)QP * n, l, c->beta(l), 0, QP, c->stream, B, d_eval, d_stride);
        launch_ntt_forward_rows(c->env, ext, c->stream);
        return;
    }
    launch_modup(c->env, S.coef, d_eval, d_stride, S.ext, (size_t)QP * n, l, c->beta(l), c->stream, B);
    launch_ntt_forward(c->env, ext, c->stream);
}

// Target limbs per fused ModUp group: the group's lifted digits stay resident in L2
// between the column kernel that writes them and the row kernel that reads them.
static int ks_group(const rk_ctx* c, int l, int B) {
    const double per_limb = (double)c->n * 8.0 * B * c->beta(l);
    const int g = (int)(c->ks_group_bytes / per_limb);
    return std::max(1, std::min(g, l + 1 + c->alpha));
}

// Inner product of the lifted input with `key` (automorphism `galois` on the lifted
// digits) into S.u [B][2][l+1+alpha][n].  `lifted` says whether S.ext already holds
// every lifted digit (hoisted rotations); otherwise the fused path lifts group by group.
static void ks_inner(rk_ctx* c, KeyRef key, int l, u64 galois, const u64* d_eval, size_t d_stride, int B, bool lifted) {
    Scratch S = scratch_layout(c);
    const int QP = l + 1 + c->alpha, beta = c->beta(l);
    const size_t es = (size_t)QP * c->n;
    if (!c->ks_fused) {
        launch_ks_inner(c->env, S.ext, es, key, S.u, l, beta, galois, c->stream, B);
        return;
    }
    if (lifted) {
        launch_ks_row(c->env, S.ext, es, d_eval, d_stride, key, S.u, l, beta, 0, QP, galois, c->stream, B);
        return;
    }
    const int G = ks_group(c, l, B);
    for (int t0 = 0; t0 < QP; t0 += G) {
        const int g = std::min(G, QP - t0);
        launch_modup_col(c->env, S.coef, S.ext, es, l, beta, t0, g, c->stream, B);
        launch_ks_row(c->env, S.ext, es, d_eval, d_stride, key, S.u, l, beta, t0, g, galois, c->stream, B);
    }
}

// ModDown of S.u and out_b = base_b + result_b (automorphism galois0 on base0), for B
// stacked inputs (base_p of member b at base_p + b * bstride); plus `addend` (the
// output's layout) when it is not null, on the staged path only.
static void ks_moddown(rk_ctx* c, int l, const u64* base0, u64 galois0, const u64* base1, size_t bstride, u64* out, size_t out_ps,
                       int B, const u64* addend = nullptr) {
    Scratch S = scratch_layout(c);
    const size_t n = c->n;
    const int QP = l + 1 + c->alpha;
    launch_ntt_inverse(c->env, LimbSet{S.u + (size_t)(l + 1) * n, (size_t)QP * n, 2 * B, c->alpha, 0, 0, c->L + 1}, c->stream);
    if (c->ks_fused) {
        RK_REQUIRE(!addend, RK_EINVAL, "fused key switching takes no addend");
        launch_moddown_col(c->env, S.u, S.w, l, c->stream, 2 * B);
        launch_moddown_row(c->env, out, out_ps, base0, galois0, base1, bstride, S.u, S.w, l, c->stream, B);
    } else {
        launch_moddown_conv(c->env, S.u, S.w, l, c->stream, 2 * B);
        launch_ntt_forward(c->env, ls_q(S.w, (size_t)(l + 1) * n, 2 * B, l + 1), c->stream);
        launch_ks_combine(c->env, out, out_ps, base0, galois0, base1, bstride, S.u, S.w, l, c->stream, B, addend);
    }
    c->n_ks += (uint64_t)B;
}

u64 galois_left(const rk_ctx* c, int r) {
    const int64_t slots = c->n / 2;
    int64_t rr = ((int64_t)r % slots + slots) % slots;
    return h_powmod(5, (u64)rr, 2ull * (u64)c->n);
}

void ev_rotate_many(rk_ctx* c, const rk_ct* a, const int* r, int k, rk_ct** outs) {
    const int l = a->level;
    const size_t ps = c->poly_stride();
    int nks = 0;
    for (int i = 0; i < k; i++) {
        RK_REQUIRE(outs[i] != a, RK_EINVAL, "rotate: output aliases input");
        RK_REQUIRE(outs[i]->B == a->B, RK_EINVAL, "rotate: stack size mismatch");
        u64 g = galois_left(c, r[i]);
        if (g != 1) {
            RK_REQUIRE(c->gal.count(g), RK_ENOKEY, "rotation key missing for r = " + std::to_string(r[i]));
            nks++;
        }
    }
    // hoisting: one ModUp serves every rotation of the list
    const u64* d = a->data + ps;
    bool lifted = false;
    if (nks > 0) {
        ks_lift(c, d, 2 * ps, l, a->B);
        if (!c->ks_fused) {
            ks_lift_ext(c, d, 2 * ps, l, a->B);
            lifted = true;
        } else if (nks > 1) {
            launch_modup_col(c->env, scratch_layout(c).coef, scratch_layout(c).ext, (size_t)(l + 1 + c->alpha) * c->n, l,
                             c->beta(l), 0, l + 1 + c->alpha, c->stream, a->B);
            lifted = true;
        }
    }
    for (int i = 0; i < k; i++) {
        u64 g = galois_left(c, r[i]);
        if (g == 1) {
            ev_copy(c, a, outs[i]);
            continue;
        }
        ks_inner(c, c->gal[g].ref(), l, g, d, 2 * ps, a->B, lifted);
        ks_moddown(c, l, a->data, g, nullptr, 2 * ps, outs[i]->data, ps, a->B);
        outs[i]->level = l;
        copy_meta(outs[i], a);
        c->n_rot += (uint64_t)a->B;
    }
}

// out = a + (a <<< r): the sum rides on the key switch's final combine (staged path).
void ev_rotate_add(rk_ctx* c, const rk_ct* a, int r, rk_ct* out) {
    RK_REQUIRE(out != a, RK_EINVAL, "rotate_add: output aliases input");
    RK_REQUIRE(out->B == a->B, RK_EINVAL, "rotate_add: stack size mismatch");
    const u64 g = galois_left(c, r);
    if (g == 1 || c->ks_fused) {
        rk_ct* outs[1] = {out};
        ev_rotate_many(c, a, &r, 1, outs);
        ev_add(c, a, out, out);
        return;
    }
    RK_REQUIRE(c->gal.count(g), RK_ENOKEY, "rotation key missing for r = " + std::to_string(r));
    const int l = a->level;
    const size_t ps = c->poly_stride();
    const u64* d = a->data + ps;
    ks_lift(c, d, 2 * ps, l, a->B);
    ks_lift_ext(c, d, 2 * ps, l, a->B);
    ks_inner(c, c->gal[g].ref(), l, g, d, 2 * ps, a->B, true);
    ks_moddown(c, l, a->data, g, nullptr, 2 * ps, out->data, ps, a->B, a->data);
    out->level = l;
    copy_meta(out, a);
    c->n_rot += (uint64_t)a->B;
}

// Member b of the stack `a` rotated left by r[b] (a different Galois element and key
// per member), plus member b of `a` when `add`: one ModUp, ModDown and NTT launch for
// the whole stack; the key inner product and the final combine run per member.
void ev_rotate_multi(rk_ctx* c, const rk_ct* a, const int* r, bool add, rk_ct* out) {
    RK_REQUIRE(out != a, RK_EINVAL, "rotate_multi: output aliases input");
    RK_REQUIRE(out->B == a->B, RK_EINVAL, "rotate_multi: stack size mismatch");
    const int B = a->B, l = a->level;
    std::vector<u64> gs(B);
    for (int b = 0; b < B; b++) {
        gs[b] = galois_left(c, r[b]);
        RK_REQUIRE(gs[b] == 1 || c->gal.count(gs[b]), RK_ENOKEY, "rotation key missing for r = " + std::to_string(r[b]));
    }
    bool all_keyed = !c->ks_fused;
    for (int b = 0; b < B; b++) all_keyed = all_keyed && gs[b] != 1;
    if (!all_keyed) {   // member by member (fused key switching, or a rotation by 0)
        for (int b = 0; b < B; b++) {
            rk_ct* ab = ct_view(a, b);
            rk_ct* ob = ct_view(out, b);
            try {
                if (add) {
                    ev_rotate_add(c, ab, r[b], ob);
                } else {
                    rk_ct* outs[1] = {ob};
                    ev_rotate_many(c, ab, &r[b], 1, outs);
                }
            } catch (...) {
                ct_free(ab);
                ct_free(ob);
                throw;
            }
            ct_free(ab);
            ct_free(ob);
        }
        out->level = l;
        copy_meta(out, a);
        return;
    }
    const size_t ps = c->poly_stride(), n = c->n;
    const int QP = l + 1 + c->alpha, beta = c->beta(l);
    const u64* d = a->data + ps;
    ks_lift(c, d, 2 * ps, l, B);
    ks_lift_ext(c, d, 2 * ps, l, B);
    Scratch S = scratch_layout(c);
    const size_t es = (size_t)QP * n;
    for (int b = 0; b < B; b++)
        launch_ks_inner(c->env, S.ext + (size_t)b * beta * es, es, c->gal[gs[b]].ref(), S.u + (size_t)b * 2 * es, l, beta, gs[b],
                        c->stream, 1);
    launch_ntt_inverse(c->env, LimbSet{S.u + (size_t)(l + 1) * n, es, 2 * B, c->alpha, 0, 0, c->L + 1}, c->stream);
    launch_moddown_conv(c->env, S.u, S.w, l, c->stream, 2 * B);
    launch_ntt_forward(c->env, ls_q(S.w, (size_t)(l + 1) * n, 2 * B, l + 1), c->stream);
    for (int b = 0; b < B; b++) {
        const u64* ab = a->data + (size_t)b * 2 * ps;
        launch_ks_combine(c->env, out->data + (size_t)b * 2 * ps, ps, ab, gs[b], nullptr, 2 * ps, S.u + (size_t)b * 2 * es,
                          S.w + (size_t)b * 2 * (l + 1) * n, l, c->stream, 1, add ? ab : nullptr);
    }
    c->n_ks += (uint64_t)B;
    c->n_rot += (uint64_t)B;
    out->level = l;
    copy_meta(out, a);
}

// Hoisted sums of rotations: for every set s and stack member b,
//   outs[s]_b = [a_b +] sum_{k < K[s]} (a_b <<< r[(s B + b) 3 + k])
// with one ModUp of the stack for all of them, the inner products of each sum added
// over Q_l P (accumulating launches), one ModDown for all the sums and a combine that
// adds the automorphic images of c0 (K[s] <= 3).  The sums' ModDown rounds once, so a
// sum equals adding its separate rotations up to that rounding.  Always on the staged
// kernels (the result does not depend on RK_OPT_KS_FUSED).
void ev_rotate_sums(rk_ctx* c, const rk_ct* a, int nsets, const int* K, const int* r, bool add, rk_ct** outs) {
    const int B = a->B, l = a->level;
    RK_REQUIRE(nsets >= 1, RK_EINVAL, "rotate_sums: no sets");
    std::vector<std::vector<u64>> gal((size_t)nsets * B);
    for (int s = 0; s < nsets; s++) {
        RK_REQUIRE(K[s] >= 1 && K[s] <= 3, RK_EINVAL, "rotate_sums: 1 to 3 rotations a sum");
        RK_REQUIRE(outs[s] != a && outs[s]->B == B, RK_EINVAL, "rotate_sums: output aliases input or stack mismatch");
        for (int b = 0; b < B; b++)
            for (int k = 0; k < K[s]; k++) {
                const int rr = r[((size_t)s * B + b) * 3 + k];
                const u64 g = galois_left(c, rr);
                RK_REQUIRE(g != 1, RK_EINVAL, "rotate_sums: rotation by 0");
                RK_REQUIRE(c->gal.count(g), RK_ENOKEY, "rotation key missing for r = " + std::to_string(rr));
                gal[(size_t)s * B + b].push_back(g);
            }
    }
    ensure_batch(c, nsets * B);   // before the lift: growing the scratch would drop it
    const size_t ps = c->poly_stride(), n = c->n;
    const u64* d = a->data + ps;
    ks_lift(c, d, 2 * ps, l, B);
    ks_lift_ext(c, d, 2 * ps, l, B);
    Scratch S = scratch_layout(c);
    const int QP = l + 1 + c->alpha, beta = c->beta(l);
    const size_t es = (size_t)QP * n;
    for (int s = 0; s < nsets; s++) {
        bool uniform = true;   // every member rotated by the same amounts: one launch for the stack
        for (int b = 1; b < B && uniform; b++) uniform = gal[(size_t)s * B + b] == gal[(size_t)s * B];
        u64* us = S.u + (size_t)s * B * 2 * es;
        if (uniform) {
            for (int k = 0; k < K[s]; k++) {
                const u64 g = gal[(size_t)s * B][k];
                launch_ks_inner(c->env, S.ext, es, c->gal[g].ref(), us, l, beta, g, c->stream, B, k > 0);
            }
        } else {
            for (int b = 0; b < B; b++)
                for (int k = 0; k < K[s]; k++) {
                    const u64 g = gal[(size_t)s * B + b][k];
                    launch_ks_inner(c->env, S.ext + (size_t)b * beta * es, es, c->gal[g].ref(), us + (size_t)b * 2 * es, l, beta,
                                    g, c->stream, 1, k > 0);
                }
        }
    }
    const int polys = 2 * nsets * B;
    launch_ntt_inverse(c->env, LimbSet{S.u + (size_t)(l + 1) * n, es, polys, c->alpha, 0, 0, c->L + 1}, c->stream);
    launch_moddown_conv(c->env, S.u, S.w, l, c->stream, polys);
    launch_ntt_forward(c->env, ls_q(S.w, (size_t)(l + 1) * n, polys, l + 1), c->stream);
    for (int s = 0; s < nsets; s++) {
        for (int b = 0; b < B; b++) {
            const std::vector<u64>& gs = gal[(size_t)s * B + b];
            GaloisSet set{(int)gs.size(), {0, 0, 0}};
            for (size_t k = 0; k < gs.size(); k++) set.g[k] = gs[k];
            const size_t m = (size_t)s * B + b;
            launch_ks_combine_sum(c->env, outs[s]->data + (size_t)b * 2 * ps, ps, a->data + (size_t)b * 2 * ps, 2 * ps, set, add,
                                  S.u + m * 2 * es, S.w + m * 2 * (l + 1) * n, l, c->stream, 1);
        }
        outs[s]->level = l;
        copy_meta(outs[s], a);
    }
    c->n_ks += (uint64_t)nsets * B;
    for (int s = 0; s < nsets; s++) c->n_rot += (uint64_t)K[s] * B;
}

// The relinearisation and rescale of B tensor products already in S.d ([B][3][l+1][n]),
// into out ([B] members at level l - 1).
static void mul_finish(rk_ctx* c, int l, int B, const rk_ct* meta, rk_ct* out) {
    Scratch S = scratch_layout(c);
    const size_t n = c->n, pl = (size_t)(l + 1) * n;
    ks_lift(c, S.d + 2 * pl, 3 * pl, l, B);
    if (!c->ks_fused) ks_lift_ext(c, S.d + 2 * pl, 3 * pl, l, B);
    ks_inner(c, c->rlk.ref(), l, 0, S.d + 2 * pl, 3 * pl, B, !c->ks_fused);
    // ModDown and rescale in one rounding: (P d_p + u_p) / (q_l P) over q_0 .. q_(l-1)
    const int QP = l + 1 + c->alpha;
    const u64 ql = c->primes[l];
    u64 pm = 1 % ql;
    for (int k = 0; k < c->alpha; k++) pm = h_mulmod(pm, c->primes[c->L + 1 + k] % ql, ql);
    launch_ks_add_pd(c->env, S.u, S.d, l, pm, shoup_companion(pm, ql), c->stream, B);
    launch_ntt_inverse(c->env, LimbSet{S.u + (size_t)l * n, (size_t)QP * n, 2 * B, c->alpha + 1, 1, l, c->L + 1}, c->stream);
    launch_moddown_rs_conv(c->env, S.u, S.w, l, c->stream, 2 * B);
    launch_ntt_forward(c->env, ls_q(S.w, (size_t)l * n, 2 * B, l), c->stream);
    launch_ks_combine_rs(c->env, out->data, c->poly_stride(), S.u, S.w, S.d, l, c->stream, B);
    out->level = l - 1;
    copy_meta(out, meta);
    c->n_ks += (uint64_t)B;
    c->n_mul += (uint64_t)B;
    c->n_rescale++;
}

void ev_mul(rk_ctx* c, const rk_ct* a, const rk_ct* b, rk_ct* out) {
    RK_REQUIRE(a->level == b->level, RK_EINVAL, "mul: level mismatch");
    RK_REQUIRE(a->B == b->B && out->B == a->B, RK_EINVAL, "mul: stack size mismatch");
    const int l = a->level, B = a->B;
    RK_REQUIRE(l >= 1, RK_EDEPTH, "mul: no level left");
    RK_REQUIRE(c->rlk.data, RK_ENOKEY, "relinearisation key missing");
    ensure_batch(c, B);
    Scratch S = scratch_layout(c);
    launch_tensor(c->env, S.d, a->data, b->data, l + 1, c->poly_stride(), c->stream, B);
    mul_finish(c, l, B, a, out);
}

// Products a[i] * b[i] of separate ciphertexts (or stacks of one size B) of one level
// as one stack: a tensor launch per pair writes members [i B, (i+1) B) of the scratch,
// then one relinearisation and rescale for all; out is a stack of n B members.
void ev_mul_pairs(rk_ctx* c, const rk_ct* const* a, const rk_ct* const* b, int n, rk_ct* out) {
    RK_REQUIRE(n >= 1, RK_EINVAL, "mul_pairs: no pairs");
    const int l = a[0]->level, B = a[0]->B;
    RK_REQUIRE(out->B == n * B, RK_EINVAL, "mul_pairs: output must hold every pair's members");
    RK_REQUIRE(l >= 1, RK_EDEPTH, "mul_pairs: no level left");
    RK_REQUIRE(c->rlk.data, RK_ENOKEY, "relinearisation key missing");
    for (int i = 0; i < n; i++)
        RK_REQUIRE(a[i]->level == l && b[i]->level == l && a[i]->B == B && b[i]->B == B, RK_EINVAL,
                   "mul_pairs: operands of one level and stack size");
    ensure_batch(c, n * B);
    Scratch S = scratch_layout(c);
    const size_t pl = (size_t)(l + 1) * c->n;
    for (int i = 0; i < n; i++)
        launch_tensor(c->env, S.d + (size_t)i * B * 3 * pl, a[i]->data, b[i]->data, l + 1, c->poly_stride(), c->stream, B);
    mul_finish(c, l, n * B, a[0], out);
}

// Times one top-level rotation with the staged key switching and with the fused
// path at three L2 group sizes (CUDA events on the context stream, zero ciphertext,
// the first rotation key) and keeps the fastest.  report: staged us, fused us at
// 24 / 48 / 96 MiB, then the choice (0 staged, else the group MiB).
void ks_autotune(rk_ctx* c, std::vector<double>& report) {
    if (c->gal.empty()) return;
    const u64 g = c->gal.begin()->first;
    int r = -1;   // a rotation amount with that Galois element
    for (int k = 1; k < c->n / 2 && r < 0; k++)
        if (galois_left(c, k) == g) r = k;
    if (r < 0) return;
    rk_ct* x = ct_alloc(c, c->L, 1);
    rk_ct* y = ct_alloc(c, c->L, 1);
    RK_CUDA(cudaMemsetAsync(x->data, 0, c->ct_words() * 8, c->stream));
    cudaEvent_t e0, e1;
    RK_CUDA(cudaEventCreate(&e0));
    RK_CUDA(cudaEventCreate(&e1));
    const bool fused0 = c->ks_fused, modup_col0 = c->modup_col;
    const double group0 = c->ks_group_bytes;
    auto time_rot = [&](bool fused, double group, bool modup_col = false) {
        c->ks_fused = fused;
        c->ks_group_bytes = group;
        c->modup_col = modup_col;
        rk_ct* outs[1] = {y};
        ev_rotate_many(c, x, &r, 1, outs);   // warm
        RK_CUDA(cudaEventRecord(e0, c->stream));
        for (int i = 0; i < 3; i++) ev_rotate_many(c, x, &r, 1, outs);
        RK_CUDA(cudaEventRecord(e1, c->stream));
        RK_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        RK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return 1000.0 * ms / 3;
    };
    try {
        const double mib = 1 << 20;
        double best = time_rot(false, group0), choice = 0;
        report.push_back(best);
        for (double gm : {24.0, 48.0, 96.0}) {
            const double t = time_rot(true, gm * mib);
            report.push_back(t);
            if (t < best) {
                best = t;
                choice = gm;
            }
        }
        report.push_back(choice);
        // the staged path with the ModUp conversion fused into the column pass
        const double t_mc = time_rot(false, group0, true);
        const bool mc = choice == 0 && t_mc < best;
        report.push_back(t_mc);
        report.push_back(mc ? 1.0 : 0.0);
        c->ks_fused = choice > 0;
        c->ks_group_bytes = choice > 0 ? choice * mib : group0;
        c->modup_col = mc;
    } catch (...) {
        c->ks_fused = fused0;
        c->ks_group_bytes = group0;
        c->modup_col = modup_col0;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ct_free(x);
        ct_free(y);
        throw;
    }
    c->n_ks -= 20;   // the timing rotations are not the caller's
    c->n_rot -= 20;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ct_free(x);
    ct_free(y);
    RK_CUDA(cudaStreamSynchronize(c->stream));
}

// ---------------------------------------------------------------------------
// Keys
// ---------------------------------------------------------------------------
static void secret_set(rk_ctx* c, const std::vector<int64_t>& s) {
    const int NP = c->n_primes;
    c->h_sk = s;
    if (!c->d_sk) RK_CUDA(rk_malloc((void**)&c->d_sk, (size_t)NP * c->n * 8));
    Scratch S = scratch_layout(c);
    upload_i64_sync(c, (int64_t*)S.misc, s.data(), c->n);
    launch_reduce_signed(c->env, (int64_t*)S.misc, ls_all(c->d_sk, 0, 1, NP), c->stream);
    launch_ntt_forward(c->env, ls_all(c->d_sk, 0, 1, NP), c->stream);
    launch_to_mont(c->env, ls_all(c->d_sk, 0, 1, NP), c->stream);
}

// small Gaussian polynomial over the first `limbs` primes, evaluation domain, into dst
static void gaussian_eval(rk_ctx* c, HostRng& rng, u64* dst, int limbs, int64_t* dev_tmp) {
    std::vector<int64_t> e(c->n);
    for (auto& x : e) x = rng.gaussian(kSigma);
    upload_i64_sync(c, dev_tmp, e.data(), c->n);
    launch_reduce_signed(c->env, dev_tmp, ls_all(dst, 0, 1, limbs), c->stream);
    launch_ntt_forward(c->env, ls_all(dst, 0, 1, limbs), c->stream);
}

static void make_pk(rk_ctx* c) {
    const int L1 = c->L + 1;
    Scratch S = scratch_layout(c);
    if (!c->d_pk) RK_CUDA(rk_malloc((void**)&c->d_pk, (size_t)2 * L1 * c->n * 8));
    HostRng rng(c->seed ^ 0x5045524B45590001ull);
    u64* a = S.misc;
    u64* e = S.misc + (size_t)L1 * c->n;
    int64_t* tmp = (int64_t*)(S.misc + (size_t)2 * L1 * c->n);
    launch_uniform(c->env, ls_all(a, 0, 1, L1), c->seed, 0xA0000000ull, c->stream);
    gaussian_eval(c, rng, e, L1, tmp);
    launch_pk(c->env, c->d_pk, (size_t)L1 * c->n, a, e, c->d_sk, L1, c->stream);
    RK_CUDA(cudaStreamSynchronize(c->stream));
}

// Switching key from s' (evaluation domain, normal form, all primes, in sp) to s.  The
// a parts are seeded: only b_j is stored, a_j is regenerated by the key switch.
static SwitchKeyDev make_switch_key(rk_ctx* c, const u64* sp, u64 stream_id) {
    const int NP = c->n_primes, L = c->L, DS = c->dsize, BL = c->beta(L);
    const size_t n = c->n;
    SwitchKeyDev key;
    key.seeded = true;
    key.seed = HostRng::mix(c->seed ^ HostRng::mix(stream_id + 0x5EED0000ull));
    cudaError_t err = rk_malloc((void**)&key.data, (size_t)BL * NP * n * 8);
    if (err != cudaSuccess) throw rk_error(RK_ENOMEM, "switching key allocation failed");
    Scratch S = scratch_layout(c);
    // misc: [sp copy is provided by caller in misc][e: NP n][tmp: n][gad: NP]
    u64* e = S.misc + (size_t)NP * n;
    int64_t* tmp = (int64_t*)(S.misc + (size_t)2 * NP * n);
    u64* gad_dev = S.misc + (size_t)2 * NP * n + n;
    HostRng rng(c->seed ^ HostRng::mix(stream_id + 0x4B4559ull));
    u64 Pmod[RK_MAX_PRIMES];
    for (int t = 0; t <= L; t++) {
        u64 pm = 1;
        for (int k = 0; k < c->alpha; k++) pm = h_mulmod(pm, c->primes[L + 1 + k] % c->primes[t], c->primes[t]);
        Pmod[t] = pm;
    }
    try {
        for (int j = 0; j < BL; j++) {
            u64* kb = key.data + (size_t)j * NP * n;
            gaussian_eval(c, rng, e, NP, tmp);
            std::vector<u64> gad(NP, 0);
            for (int t = j * DS; t < std::min((j + 1) * DS, L + 1); t++) gad[t] = h_mulmod(Pmod[t], c->h_pc[t].r_mod, c->primes[t]);
            RK_CUDA(cudaMemcpyAsync(gad_dev, gad.data(), NP * 8, cudaMemcpyHostToDevice, c->stream));
            launch_key_digit_seeded(c->env, kb, e, c->d_sk, sp, gad_dev, key.seed, j, NP, c->stream);
            RK_CUDA(cudaStreamSynchronize(c->stream));
        }
    } catch (...) {
        cudaFree(key.data);
        throw;
    }
    return key;
}

static void set_key(SwitchKeyDev& slot, const SwitchKeyDev& key) {
    if (slot.data) cudaFree(slot.data);
    slot = key;
}

static void make_relin_key(rk_ctx* c) {
    Scratch S = scratch_layout(c);
    launch_square_secret(c->env, S.misc, c->d_sk, c->n_primes, c->stream);
    const SwitchKeyDev k = make_switch_key(c, S.misc, 1);
    set_key(c->rlk, k);
    c->generation++;
}

void keys_add_rotations(rk_ctx* c, const std::vector<int>& rotations) {
    RK_REQUIRE(c->d_sk, RK_EINVAL, "no secret key");
    Scratch S = scratch_layout(c);
    const int NP = c->n_primes;
    for (int r : rotations) {
        u64 g = galois_left(c, r);
        if (g == 1 || c->gal.count(g)) continue;
        // s' = sigma_g(s): from Montgomery form, then permute evaluations
        u64* s_norm = S.misc + (size_t)2 * NP * c->n + 2 * c->n;   // beyond make_switch_key's area
        launch_from_mont(c->env, s_norm, c->d_sk, NP, c->stream);
        launch_automorph(c->env, S.misc, s_norm, g, NP, c->stream);
        c->gal[g] = make_switch_key(c, S.misc, 16 + g);
    }
}

void keys_generate(rk_ctx* c, uint64_t seed, const std::vector<int>& rotations) {
    c->seed = seed;
    HostRng rng(seed ^ 0x5345435245540001ull);
    std::vector<int64_t> s(c->n);
    for (auto& x : s) x = rng.ternary();
    secret_set(c, s);
    make_pk(c);
    make_relin_key(c);
    keys_add_rotations(c, rotations);
}

void secret_import(rk_ctx* c, const int64_t* s, size_t n) {
    RK_REQUIRE(n == (size_t)c->n, RK_EINVAL, "secret length must be n");
    for (size_t i = 0; i < n; i++) RK_REQUIRE(s[i] >= -1 && s[i] <= 1, RK_EINVAL, "secret must be ternary");
    if (c->seed == 0) c->seed = 0x1234567ull;
    secret_set(c, std::vector<int64_t>(s, s + n));
    make_pk(c);
}

// Switching key words: [beta_L][parts][L+1+alpha][n], parts 2 (b_j, a_j) or 1 (b_j
// of a seeded key), coefficient domain, residues in [0, q).
void key_import(rk_ctx* c, uint32_t kind, uint64_t galois, const uint64_t* coeffs, size_t words, bool seeded, uint64_t seed) {
    const int NP = c->n_primes, BL = c->beta(c->L), parts = seeded ? 1 : 2;
    const size_t n = c->n, expect = (size_t)BL * parts * NP * n;
    RK_REQUIRE(words == expect, RK_EINVAL, "key size mismatch: expected " + std::to_string(expect) + " words");
    RK_REQUIRE(kind == RK_KEY_RELIN || kind == RK_KEY_GALOIS, RK_EINVAL, "bad key kind");
    for (int t = 0; t < NP; t++)  // spot-check residues are canonical
        RK_REQUIRE(coeffs[(size_t)t * n] < c->primes[t], RK_EFORMAT, "key residue out of range");
    SwitchKeyDev key;
    key.seeded = seeded;
    key.seed = seed;
    RK_CUDA(rk_malloc((void**)&key.data, expect * 8));
    RK_CUDA(cudaMemcpyAsync(key.data, coeffs, expect * 8, cudaMemcpyHostToDevice, c->stream));
    launch_ntt_forward(c->env, ls_all(key.data, (size_t)NP * n, BL * parts, NP), c->stream);
    launch_to_mont(c->env, ls_all(key.data, (size_t)NP * n, BL * parts, NP), c->stream);
    RK_CUDA(cudaStreamSynchronize(c->stream));
    c->generation++;
    set_key(kind == RK_KEY_RELIN ? c->rlk : c->gal[galois], key);
}

size_t key_words(const rk_ctx* c, const SwitchKeyDev& key) {
    return (size_t)c->beta(c->L) * (key.seeded ? 1 : 2) * c->n_primes * c->n;
}

// A switching key in key_import's layout (coefficient domain, plain residues).
void key_export(rk_ctx* c, const SwitchKeyDev& key, u64* host_out) {
    const int NP = c->n_primes;
    const size_t n = c->n, words = key_words(c, key);
    const int polys = (int)(words / ((size_t)NP * n));
    u64* tmp = nullptr;
    RK_CUDA(rk_malloc_async((void**)&tmp, words * 8, c->stream));
    for (int p = 0; p < polys; p++) launch_from_mont(c->env, tmp + (size_t)p * NP * n, key.data + (size_t)p * NP * n, NP, c->stream);
    launch_ntt_inverse(c->env, ls_all(tmp, (size_t)NP * n, polys, NP), c->stream);
    RK_CUDA(cudaMemcpyAsync(host_out, tmp, words * 8, cudaMemcpyDeviceToHost, c->stream));
    RK_CUDA(cudaFreeAsync(tmp, c->stream));
    RK_CUDA(cudaStreamSynchronize(c->stream));
}

// ---------------------------------------------------------------------------
// Client operations
// ---------------------------------------------------------------------------
rk_ct* encrypt_values(rk_ctx* c, const double* v, uint32_t count, uint32_t N, uint32_t Q, uint32_t n_real) {
    RK_REQUIRE(c->d_pk, RK_EINVAL, "no public key: call rk_keygen or rk_secret_import first");
    const size_t slots = c->n / 2;
    RK_REQUIRE(N >= 1 && (N & (N - 1)) == 0, RK_EINVAL, "N must be a power of two");
    RK_REQUIRE(n_real >= 1 && n_real <= N, RK_EINVAL, "n_real must be in [1, N]");
    RK_REQUIRE(Q >= 1 && (size_t)Q * N * N <= slots, RK_EINVAL, "Q * N^2 exceeds the slot count");
    RK_REQUIRE(count <= (size_t)Q * n_real, RK_EINVAL, "more values than Q * n_real");
    std::vector<double> z(slots, 0.0);
    for (uint32_t i = 0; i < count; i++) {
        RK_REQUIRE(v[i] >= 0.0 && v[i] < 1.0, RK_EINVAL, "values must lie in [0, 1)");
        z[(size_t)(i / n_real) * N * N + (i % n_real)] = v[i];
    }
    std::vector<double> u;
    encode_unscaled(c->log_n, z.data(), z.size(), u);
    const int L1 = c->L + 1;
    const size_t n = c->n;
    std::vector<int64_t> host(4 * n);
    HostRng rng(c->seed ^ HostRng::mix(0x454E43ull + c->enc_counter++));
    for (size_t k = 0; k < n; k++) host[k] = rng.ternary();
    for (size_t k = 0; k < n; k++) host[n + k] = rng.gaussian(kSigma);
    for (size_t k = 0; k < n; k++) host[2 * n + k] = rng.gaussian(kSigma);
    for (size_t k = 0; k < n; k++) host[3 * n + k] = round_half_away(c->scales[c->L] * u[k]);
    Scratch S = scratch_layout(c);
    int64_t* tmp2 = (int64_t*)S.u;   // 2 (L+1+alpha) n >= 4 n words
    upload_i64_sync(c, tmp2, host.data(), 4 * n);
    LimbSet r = ls_q(S.misc, (size_t)L1 * n, 4, L1);
    launch_reduce_signed(c->env, tmp2, r, c->stream);
    launch_ntt_forward(c->env, r, c->stream);
    rk_ct* ct = ct_alloc(c, c->L);
    launch_encrypt(c->env, ct->data, c->poly_stride(), S.misc, c->d_pk, (size_t)L1 * n, L1, c->stream);
    ct->N = N;
    ct->Q = Q;
    ct->n_real = n_real;
    ct->layout = RK_LAYOUT_ROW;
    return ct;
}

void decrypt_slots(rk_ctx* c, const rk_ct* ct, std::vector<double>& slots) {
    RK_REQUIRE(c->d_sk, RK_EINVAL, "no secret key");
    RK_REQUIRE(ct->B == 1, RK_EINVAL, "decrypt a stacked handle after rk_ct_unstack");
    const int l = ct->level;
    const size_t n = c->n;
    Scratch S = scratch_layout(c);
    launch_decrypt(c->env, S.misc, ct->data, ct->data + c->poly_stride(), c->d_sk, l + 1, c->stream);
    launch_ntt_inverse(c->env, ls_q(S.misc, 0, 1, l + 1), c->stream);
    const int use = l >= 1 ? 2 : 1;
    std::vector<u64> h((size_t)use * n);
    RK_CUDA(cudaMemcpyAsync(h.data(), S.misc, (size_t)use * n * 8, cudaMemcpyDeviceToHost, c->stream));
    RK_CUDA(cudaStreamSynchronize(c->stream));
    std::vector<double> m(n);
    const u64 q0 = c->primes[0];
    if (use == 1) {
        for (size_t k = 0; k < n; k++) {
            u64 x = h[k];
            m[k] = x > q0 / 2 ? -(double)(q0 - x) : (double)x;
        }
    } else {
        const u64 q1 = c->primes[1];
        const u64 q0inv = h_invmod(q0 % q1, q1);
        const u128 Q = (u128)q0 * q1;
        for (size_t k = 0; k < n; k++) {
            u64 x0 = h[k], x1 = h[n + k];
            u64 t = h_mulmod((x1 + q1 - (x0 % q1)) % q1, q0inv, q1);
            u128 x = (u128)x0 + (u128)q0 * t;
            m[k] = x > Q / 2 ? -(double)(Q - x) : (double)x;
        }
    }
    for (size_t k = 0; k < n; k++) m[k] /= c->scales[l];
    decode_coeffs(c->log_n, m, slots);
}

rk_ct* ct_import(rk_ctx* c, const uint64_t* coeffs, int level) {
    RK_REQUIRE(level >= 0 && level <= c->L, RK_EINVAL, "bad level");
    const size_t n = c->n, pl = (size_t)(level + 1) * n;
    for (int t = 0; t <= level; t++)
        RK_REQUIRE(coeffs[(size_t)t * n] < c->primes[t] && coeffs[pl + (size_t)t * n] < c->primes[t], RK_EFORMAT,
                   "ciphertext residue out of range");
    rk_ct* ct = ct_alloc(c, level);
    RK_CUDA(cudaMemcpyAsync(ct->data, coeffs, pl * 8, cudaMemcpyHostToDevice, c->stream));
    RK_CUDA(cudaMemcpyAsync(ct->data + c->poly_stride(), coeffs + pl, pl * 8, cudaMemcpyHostToDevice, c->stream));
    launch_ntt_forward(c->env, ls_q(ct->data, c->poly_stride(), 2, level + 1), c->stream);
    RK_CUDA(cudaStreamSynchronize(c->stream));
    return ct;
}

void ct_export(rk_ctx* c, const rk_ct* ct, uint64_t* coeffs) {
    RK_REQUIRE(ct->B == 1, RK_EINVAL, "export a stacked handle after rk_ct_unstack");
    const int l = ct->level;
    const size_t n = c->n, pl = (size_t)(l + 1) * n;
    Scratch S = scratch_layout(c);
    RK_CUDA(cudaMemcpyAsync(S.misc, ct->data, pl * 8, cudaMemcpyDeviceToDevice, c->stream));
    RK_CUDA(cudaMemcpyAsync(S.misc + pl, ct->data + c->poly_stride(), pl * 8, cudaMemcpyDeviceToDevice, c->stream));
    launch_ntt_inverse(c->env, ls_q(S.misc, pl, 2, l + 1), c->stream);
    RK_CUDA(cudaMemcpyAsync(coeffs, S.misc, 2 * pl * 8, cudaMemcpyDeviceToHost, c->stream));
    RK_CUDA(cudaStreamSynchronize(c->stream));
}
