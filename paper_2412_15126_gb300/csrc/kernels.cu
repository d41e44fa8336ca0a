// CUDA kernels of the RNS-CKKS evaluator (sm_103a).
//
// Data: residue polynomials of n = 2^log_n 64-bit words, limb-major, in the
// evaluation (NTT) domain unless a kernel says otherwise.  Evaluation order of the
// forward NTT: index i holds the value at psi^(2 brev(i) + 1), psi the chosen
// primitive 2n-th root of unity modulo the limb's prime.
#include <algorithm>

#include "ntt_core.cuh"

#define TPB 256

const char* const kKernelKindNames[KK_COUNT] = {"ntt_fwd", "ntt_inv", "modup", "ks_inner", "moddown_conv",
                                               "ks_combine", "tensor", "rescale", "pointwise", "client"};

// ===========================================================================
// Pointwise kernels on ciphertexts (layout [2][L+1][n], limb t <-> q_t).
// Two consecutive coefficients a thread, moved as one 16-byte access (every offset
// below is even and every buffer 16-byte aligned); grid: (n / (2 TPB), limbs, polys).
// ===========================================================================
__device__ __forceinline__ ulonglong2 ld2(const u64* p) { return *reinterpret_cast<const ulonglong2*>(p); }
__device__ __forceinline__ void st2(u64* p, u64 x, u64 y) { *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(x, y); }
inline dim3 grid2(const KernelEnv& env, int limbs, int polys) { return dim3(env.n / (2 * TPB), limbs, polys); }

__global__ void k_addsub(u64* out, const u64* a, const u64* b, int n, size_t ps, const PrimeConst* __restrict__ pc, int mode) {
    RK_KERNEL_PROLOGUE();
    const int k = 2 * (blockIdx.x * TPB + threadIdx.x), t = blockIdx.y, c = blockIdx.z;
    const u64 q = pc[t].q;
    const size_t off = c * ps + (size_t)t * n + k;
    const ulonglong2 x = ld2(a + off);
    if (mode == 2) {
        st2(out + off, x.x ? q - x.x : 0, x.y ? q - x.y : 0);
        return;
    }
    const ulonglong2 y = ld2(b + off);
    if (mode == 0) st2(out + off, add_mod(x.x, y.x, q), add_mod(x.y, y.y, q));
    else st2(out + off, sub_mod(x.x, y.x, q), sub_mod(x.y, y.y, q));
}

void launch_addsub(const KernelEnv& env, u64* out, const u64* a, const u64* b, int limbs, size_t ps, int mode, cudaStream_t st,
                   int polys) {
    ProfScope pf(env, KK_POINTWISE, st, 1, 3.0 * polys * limbs * 8.0 * env.n, 0.0);
    rk_launch(k_addsub, grid2(env, limbs, polys), TPB, 0, st, out, a, b, env.n, ps, env.pc, mode);
}

// out0 = a0 + K_t, out1 = a1
__global__ void k_add_const(u64* out, const u64* a, ScalarArg K, int n, size_t ps, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = 2 * (blockIdx.x * TPB + threadIdx.x), t = blockIdx.y, c = blockIdx.z;
    const size_t off = c * ps + (size_t)t * n + k;
    ulonglong2 x = ld2(a + off);
    if ((c & 1) == 0) {
        const u64 q = pc[t].q;
        x.x = add_mod(x.x, K.w[t], q);
        x.y = add_mod(x.y, K.w[t], q);
    }
    st2(out + off, x.x, x.y);
}

void launch_add_const(const KernelEnv& env, u64* out, const u64* a, const ScalarArg& K, int limbs, size_t ps, cudaStream_t st,
                      int polys) {
    ProfScope pf(env, KK_POINTWISE, st, 1, 2.0 * polys * limbs * 8.0 * env.n, 0.0);
    rk_launch(k_add_const, grid2(env, limbs, polys), TPB, 0, st, out, a, K, env.n, ps, env.pc);
}

// out = a * K_t (Shoup)
// limbs t0 .. t0 + gridDim.y - 1
__global__ void k_mul_scalar(u64* out, const u64* a, ScalarArg K, int n, size_t ps, int t0, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = 2 * (blockIdx.x * TPB + threadIdx.x), t = blockIdx.y + t0, c = blockIdx.z;
    const size_t off = c * ps + (size_t)t * n + k;
    const u64 q = pc[t].q;
    const ulonglong2 x = ld2(a + off);
    st2(out + off, shoup_mul(x.x, K.w[t], K.wsh[t], q), shoup_mul(x.y, K.w[t], K.wsh[t], q));
}

void launch_mul_scalar(const KernelEnv& env, u64* out, const u64* a, const ScalarArg& K, int limbs, size_t ps, cudaStream_t st,
                       int polys, int t0) {
    ProfScope pf(env, KK_POINTWISE, st, 1, 2.0 * polys * limbs * 8.0 * env.n, 1.0 * polys * limbs * env.n);
    rk_launch(k_mul_scalar, grid2(env, limbs, polys), TPB, 0, st, out, a, K, env.n, ps, t0, env.pc);
}

// out = a * pt, pt stored times R ([limbs][n])
__global__ void k_mul_plain(u64* out, const u64* a, const u64* pt, int n, size_t ps, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = 2 * (blockIdx.x * TPB + threadIdx.x), t = blockIdx.y, c = blockIdx.z;
    const size_t off = c * ps + (size_t)t * n + k;
    const PrimeConst P = pc[t];
    const ulonglong2 x = ld2(a + off), m = ld2(pt + (size_t)t * n + k);
    st2(out + off, mont_mul(x.x, m.x, P.q, P.qinv), mont_mul(x.y, m.y, P.q, P.qinv));
}

void launch_mul_plain(const KernelEnv& env, u64* out, const u64* a, const u64* pt, int limbs, size_t ps, cudaStream_t st,
                      int polys) {
    ProfScope pf(env, KK_POINTWISE, st, 1, (2.0 * polys + 1.0) * limbs * 8.0 * env.n, 1.0 * polys * limbs * env.n);
    rk_launch(k_mul_plain, grid2(env, limbs, polys), TPB, 0, st, out, a, pt, env.n, ps, env.pc);
}

// out (+)= sum_i x_i * K_i, exact modular arithmetic, one reduction per output
__global__ void k_lincomb(u64* out, LincombArg a, int terms, int accumulate, int n, size_t ps, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = 2 * (blockIdx.x * TPB + threadIdx.x), t = blockIdx.y, c = blockIdx.z;
    const PrimeConst P = pc[t];
    const size_t off = c * ps + (size_t)t * n + k;
    Acc128 acc0, acc1;
    for (int i = 0; i < terms; i++) {
        const ulonglong2 x = ld2(a.x[i] + off);
        acc0.mac(x.x, a.KR[i][t]);
        acc1.mac(x.y, a.KR[i][t]);
    }
    u64 r0 = acc0.redc(P.q, P.qinv), r1 = acc1.redc(P.q, P.qinv);
    if (accumulate) {
        const ulonglong2 o = ld2(out + off);
        r0 = add_mod(r0, o.x, P.q);
        r1 = add_mod(r1, o.y, P.q);
    }
    st2(out + off, r0, r1);
}

void launch_lincomb(const KernelEnv& env, u64* out, const LincombArg& a, int terms, bool accumulate, int limbs, size_t ps,
                    cudaStream_t st, int polys) {
    ProfScope pf(env, KK_POINTWISE, st, 1, (terms + 1.0) * polys * limbs * 8.0 * env.n, 1.0 * terms * polys * limbs * env.n);
    rk_launch(k_lincomb, grid2(env, limbs, polys), TPB, 0, st, out, a, terms, accumulate ? 1 : 0, env.n, ps, env.pc);
}

// d = [d0 | d1 | d2] each [limbs][n]: d0 = x0 y0, d1 = x0 y1 + x1 y0, d2 = x1 y1
// one ciphertext pair per blockIdx.z (stacked layout [B][2][L+1][n]); d is [B][3][limbs][n]
template <bool SP>
__global__ void k_tensor(u64* d, const u64* x, const u64* y, int limbs, int n, size_t ps, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = 2 * (blockIdx.x * TPB + threadIdx.x), t = blockIdx.y, b = blockIdx.z;
    const PrimeConst P = pc[t];
    const size_t pl = (size_t)limbs * n;
    x += (size_t)b * 2 * ps;
    y += (size_t)b * 2 * ps;
    d += (size_t)b * 3 * pl;
    const size_t off = (size_t)t * n + k;
    const ulonglong2 X0 = ld2(x + off), X1 = ld2(x + ps + off), Y0 = ld2(y + off), Y1 = ld2(y + ps + off);
    u64 r[3][2];
    const u64 x0s[2] = {X0.x, X0.y}, x1s[2] = {X1.x, X1.y}, y0s[2] = {Y0.x, Y0.y}, y1s[2] = {Y1.x, Y1.y};
#pragma unroll
    for (int e = 0; e < 2; e++) {
        const u64 x0 = x0s[e], x1 = x1s[e], y0 = y0s[e], y1 = y1s[e];
        Acc128 a1;
        a1.mac(x0, y1);
        a1.mac(x1, y0);
        r[0][e] = shoup_mul(mont_mul_t<SP>(x0, y0, P.q, P.qinv), P.r_mod, P.r_shoup, P.q);
        r[1][e] = shoup_mul(a1.template redc_t<SP>(P.q, P.qinv), P.r_mod, P.r_shoup, P.q);
        r[2][e] = shoup_mul(mont_mul_t<SP>(x1, y1, P.q, P.qinv), P.r_mod, P.r_shoup, P.q);
    }
    st2(d + off, r[0][0], r[0][1]);
    st2(d + pl + off, r[1][0], r[1][1]);
    st2(d + 2 * pl + off, r[2][0], r[2][1]);
}

void launch_tensor(const KernelEnv& env, u64* d, const u64* x, const u64* y, int limbs, size_t ps, cudaStream_t st, int B) {
    ProfScope pf(env, KK_TENSOR, st, 1, 7.0 * B * limbs * 8.0 * env.n, 4.0 * B * limbs * env.n);
    if (env.sp)
        rk_launch(k_tensor<true>, grid2(env, limbs, B), TPB, 0, st, d, x, y, limbs, env.n, ps, env.pc);
    else
        rk_launch(k_tensor<false>, grid2(env, limbs, B), TPB, 0, st, d, x, y, limbs, env.n, ps, env.pc);
}

// ===========================================================================
// Basis conversion (coefficient domain).
// ===========================================================================
// ModUp of every digit: ext[j][t][k], t over Q_l u P (QP limb order).
// The digit's own limbs are copied from the evaluation-domain input x_eval (the
// conversion reproduces them exactly), so the following NTT can skip them.
// Each thread converts CONV_EL coefficients (k0 + e TPB) so that every conversion
// constant, staged in shared memory, serves CONV_EL products.
#ifndef CONV_EL   // a build may set another width
#define CONV_EL 4
#endif
template <int DS, bool SP>
__global__ void __launch_bounds__(TPB) k_modup(const u64* __restrict__ x, const u64* __restrict__ x_eval, u64* __restrict__ ext,
                                               size_t ext_stride, int level, int L, int alpha, ConvTables cv, int n,
                                               const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    __shared__ u64 s_c[DS * RK_MAX_PRIMES];             // (D/q_i) R mod prime(t), [i][t]
    __shared__ u64 s_q[RK_MAX_PRIMES], s_qinv[RK_MAX_PRIMES];
    const int j = blockIdx.y;
    const int lo = j * DS, hi = min(lo + DS, level + 1), ns = hi - lo;
    const u64* tab = cv.modup + ((size_t)level * cv.beta_max + j) * cv.modup_stride;
    const int T = L + 1 + alpha;
    const int limbs = level + 1 + alpha;
    // grid z splits the target limbs into groups (more blocks for the same work)
    const int chunk = (limbs + gridDim.z - 1) / gridDim.z;
    const int t0 = blockIdx.z * chunk, t1 = min(limbs, t0 + chunk);
    for (int idx = threadIdx.x; idx < ns * limbs; idx += TPB) {
        const int i = idx / limbs, t = idx - i * limbs;
        if (t >= t0 && t < t1) s_c[i * RK_MAX_PRIMES + t] = tab[2 * DS + (size_t)i * T + t];
    }
    for (int t = t0 + threadIdx.x; t < t1; t += TPB) {
        const int pid = t <= level ? t : L + 1 + (t - level - 1);
        s_q[t] = pc[pid].q;
        s_qinv[t] = pc[pid].qinv;
    }
    __syncthreads();
    const int k0 = blockIdx.x * (TPB * CONV_EL) + threadIdx.x;
    u64 y[CONV_EL][DS];
#pragma unroll
    for (int i = 0; i < DS; i++) {
        if (i < ns) {
            const u64 qi = pc[lo + i].q, w = tab[i], wsh = tab[DS + i];
            const u64* xi = x + (size_t)(lo + i) * n + k0;
#pragma unroll
            for (int e = 0; e < CONV_EL; e++) y[e][i] = shoup_mul(xi[e * TPB], w, wsh, qi);
        }
    }
    for (int t = t0; t < t1; t++) {
        u64* out = ext + (size_t)j * ext_stride + (size_t)t * n + k0;
        if (t >= lo && t < hi) {
            const u64* xe = x_eval + (size_t)t * n + k0;
#pragma unroll
            for (int e = 0; e < CONV_EL; e++) out[e * TPB] = xe[e * TPB];
            continue;
        }
        Acc128 acc[CONV_EL];
#pragma unroll
        for (int i = 0; i < DS; i++) {
            if (i < ns) {
                const u64 cst = s_c[i * RK_MAX_PRIMES + t];
#pragma unroll
                for (int e = 0; e < CONV_EL; e++) acc[e].mac(y[e][i], cst);
            }
        }
        const u64 q = s_q[t], qinv = s_qinv[t];
#pragma unroll
        for (int e = 0; e < CONV_EL; e++) out[e * TPB] = acc[e].template redc_t<SP>(q, qinv);
    }
}

// B stacked inputs: x is [B][l+1][n] (coefficient domain), x_eval_b = x_eval + b * eval_stride
// (evaluation domain), ext is [B][beta][l+1+alpha][n] (ext_stride per digit)
void launch_modup(const KernelEnv& env, const u64* x, const u64* x_eval, size_t eval_stride, u64* ext, size_t ext_stride,
                  int level, int beta, cudaStream_t st, int B) {
    ProfScope pf(env, KK_MODUP, st, B, B * (2.0 * (level + 1) + (double)beta * (level + 1 + env.alpha)) * 8.0 * env.n,
                 (double)B * (level + 1 + env.alpha) * (level + 1) * env.n);
    // about eight blocks an SM: the target limbs split over grid z when the digits'
    // coefficient blocks alone would leave a ragged last wave
    const int bxy = env.n / (TPB * CONV_EL) * beta, limbs = level + 1 + env.alpha;
    const int nz = std::max(1, std::min(limbs, (8 * env.sms + bxy - 1) / bxy));
    dim3 g(env.n / (TPB * CONV_EL), beta, nz);
    for (int b = 0; b < B; b++) {
        const u64* xb = x + (size_t)b * (level + 1) * env.n;
        const u64* eb = x_eval + (size_t)b * eval_stride;
        u64* ob = ext + (size_t)b * beta * ext_stride;
        switch (env.conv.dsize) {
#define RK_MODUP_CASE(D)                                                                                                 \
    case D:                                                                                                              \
        if (env.sp)                                                                                                      \
            rk_launch(k_modup<D, true>, g, TPB, 0, st, xb, eb, ob, ext_stride, level, env.L, env.alpha, env.conv, env.n,  \
                      env.pc);                                                                                           \
        else                                                                                                             \
            rk_launch(k_modup<D, false>, g, TPB, 0, st, xb, eb, ob, ext_stride, level, env.L, env.alpha, env.conv, env.n, \
                      env.pc);                                                                                           \
        break;
            RK_MODUP_CASE(1) RK_MODUP_CASE(2) RK_MODUP_CASE(3) RK_MODUP_CASE(4)
            RK_MODUP_CASE(5) RK_MODUP_CASE(6) RK_MODUP_CASE(7) RK_MODUP_CASE(8)
#undef RK_MODUP_CASE
            default: throw rk_error(RK_EINVAL, "digit size out of range");
        }
    }
}

// ModDown conversion of the P part of u ([2][l+1+alpha][n], P limbs already in the
// coefficient domain) to w = [2][l+1][n]; CONV_EL coefficients a thread.  Each term
// y_k is centred on its own (the multiple of S is the count of terms above s_k / 2).
// RS (a product's ModDown fused with its rescale): the sources are limbs l .. l+alpha
// (q_l then the P limbs, coefficient domain), S = q_l P, w = [2][l][n], and the
// multiple of S is decided by one rounding, v = floor(sum_k y_k (1/s_k) + 1/2) in
// IEEE double (products and sums rounded to nearest in source order), so that w is the
// centred residue of u mod S and the product is round(u / S).
template <int A, bool RS, bool SP>
__global__ void __launch_bounds__(TPB) k_moddown_conv(const u64* __restrict__ u, u64* __restrict__ w, int level, int L,
                                                      ConvTables cv, int n, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    constexpr int NS = A + (RS ? 1 : 0);
    __shared__ u64 s_c[NS * RK_MAX_PRIMES];     // (S/s_k) R mod q_i, [k][i]
    __shared__ u64 s_q[RK_MAX_PRIMES], s_qinv[RK_MAX_PRIMES], s_pm[RK_MAX_PRIMES];
    const int c = blockIdx.y;
    const int nt = RS ? level : level + 1;   // target limbs
    // grid z splits the target limbs into groups of `chunk` (each block recomputes the
    // few centred source terms, so that small sets still fill the device)
    const int chunk = (nt + gridDim.z - 1) / gridDim.z;
    const int i0 = blockIdx.z * chunk, i1 = min(nt, i0 + chunk);
    const u64* blk = RS ? cv.mdrs + (size_t)level * cv.mdrs_stride : cv.moddown;
    const u64* cm = blk + 2 * NS;
    const u64* pmod = cm + (size_t)NS * (L + 1);
    for (int idx = threadIdx.x; idx < NS * nt; idx += TPB) {
        const int kk = idx / nt, i = idx - kk * nt;
        if (i >= i0 && i < i1) s_c[kk * RK_MAX_PRIMES + i] = cm[(size_t)kk * (L + 1) + i];
    }
    for (int i = i0 + threadIdx.x; i < i1; i += TPB) {
        s_q[i] = pc[i].q;
        s_qinv[i] = pc[i].qinv;
        s_pm[i] = pmod[i];
    }
    __syncthreads();
    const int ul = level + 1 + A;
    const int k0 = blockIdx.x * (TPB * CONV_EL) + threadIdx.x;
    const u64* up = u + (size_t)c * ul * n + (size_t)(RS ? level : level + 1) * n + k0;
    // centred terms: y_k in (-s_k/2, s_k/2]; a negative term contributes y_k (S/s_k) - S
    u64 y[CONV_EL][NS];
    int nneg[CONV_EL];
    double f[CONV_EL];
    const double* rcp = reinterpret_cast<const double*>(pmod + 3 * (L + 1));
#pragma unroll
    for (int e = 0; e < CONV_EL; e++) {
        nneg[e] = 0;
        f[e] = 0.0;
    }
#pragma unroll
    for (int kk = 0; kk < NS; kk++) {
        const u64 sk = RS ? (kk == 0 ? pc[level].q : pc[L + kk].q) : pc[L + 1 + kk].q;
        const u64 iv = blk[kk], ivsh = blk[NS + kk];
#pragma unroll
        for (int e = 0; e < CONV_EL; e++) {
            y[e][kk] = shoup_mul(up[(size_t)kk * n + e * TPB], iv, ivsh, sk);
            if (RS)
                f[e] = __dadd_rn(f[e], __dmul_rn(__ull2double_rn(y[e][kk]), rcp[kk]));
            else
                nneg[e] += y[e][kk] > (sk >> 1) ? 1 : 0;
        }
    }
    if (RS) {
#pragma unroll
        for (int e = 0; e < CONV_EL; e++) nneg[e] = (int)floor(__dadd_rn(f[e], 0.5));
    }
    u64* out = w + (size_t)c * nt * n + k0;
    for (int i = i0; i < i1; i++) {
        const u64 q = s_q[i], qinv = s_qinv[i], pm = s_pm[i];
        Acc128 acc[CONV_EL];
#pragma unroll
        for (int kk = 0; kk < NS; kk++) {
            const u64 cst = s_c[kk * RK_MAX_PRIMES + i];
#pragma unroll
            for (int e = 0; e < CONV_EL; e++) acc[e].mac(y[e][kk], cst);
        }
#pragma unroll
        for (int e = 0; e < CONV_EL; e++) {
            u64 r = acc[e].template redc_t<SP>(q, qinv);
            for (int z = 0; z < nneg[e]; z++) r = sub_mod(r, pm, q);
            out[(size_t)i * n + e * TPB] = r;
        }
    }
}

template <bool RS>
static void moddown_conv_launch(const KernelEnv& env, const u64* u, u64* w, int level, cudaStream_t st, int polys) {
    const int nt = RS ? level : level + 1, ns = env.alpha + (RS ? 1 : 0);
    ProfScope pf(env, KK_MODDOWN, st, 1, polys * (1.0 * ns + nt) * 8.0 * env.n, 1.0 * polys * nt * ns * env.n);
    // enough blocks for two waves: the target limbs split over grid z when the
    // coefficient blocks of the polynomials alone would leave SMs idle
    const int bxy = env.n / (TPB * CONV_EL) * polys;
    const int nz = std::max(1, std::min(nt, (2 * env.sms + bxy - 1) / bxy));
    dim3 g(env.n / (TPB * CONV_EL), polys, nz);
    switch (env.alpha) {
#define RK_MD_CASE(A)                                                                               \
    case A:                                                                                         \
        if (env.sp)                                                                                 \
            rk_launch(k_moddown_conv<A, RS, true>, g, TPB, 0, st, u, w, level, env.L, env.conv, env.n, env.pc);  \
        else                                                                                        \
            rk_launch(k_moddown_conv<A, RS, false>, g, TPB, 0, st, u, w, level, env.L, env.conv, env.n, env.pc); \
        break;
        RK_MD_CASE(1) RK_MD_CASE(2) RK_MD_CASE(3) RK_MD_CASE(4) RK_MD_CASE(5) RK_MD_CASE(6) RK_MD_CASE(7) RK_MD_CASE(8)
#undef RK_MD_CASE
        default: throw rk_error(RK_EINVAL, "special prime count out of range");
    }
}

void launch_moddown_conv(const KernelEnv& env, const u64* u, u64* w, int level, cudaStream_t st, int polys) {
    moddown_conv_launch<false>(env, u, w, level, st, polys);
}

void launch_moddown_rs_conv(const KernelEnv& env, const u64* u, u64* w, int level, cudaStream_t st, int polys) {
    moddown_conv_launch<true>(env, u, w, level, st, polys);
}

// Limb l of a product's inner products gains P d (d the tensor's d_0 / d_1, evaluation
// domain): u_c[l] += (P mod q_l) d_p[l], c = 2b + p.  grid (n/TPB, 1, 2B)
__global__ void k_ks_add_pd(u64* u, const u64* d, int level, int alpha, u64 pm, u64 pm_sh, int n,
                            const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = blockIdx.x * TPB + threadIdx.x, c = blockIdx.z;
    const int b = c >> 1, p = c & 1;
    const size_t pl = (size_t)(level + 1) * n;
    const u64 q = pc[level].q;
    u64* up = u + (size_t)c * (level + 1 + alpha) * n + (size_t)level * n + k;
    const u64 dv = d[(size_t)b * 3 * pl + (size_t)p * pl + (size_t)level * n + k];
    *up = add_mod(*up, shoup_mul(dv, pm, pm_sh, q), q);
}

void launch_ks_add_pd(const KernelEnv& env, u64* u, const u64* d, int level, u64 pm, u64 pm_sh, cudaStream_t st, int B) {
    ProfScope pf(env, KK_KS_COMBINE, st, 1, 3.0 * 2 * B * 8.0 * env.n, 2.0 * B * env.n);
    dim3 g(env.n / TPB, 1, 2 * B);
    rk_launch(k_ks_add_pd, g, TPB, 0, st, u, d, level, env.alpha, pm, pm_sh, env.n, env.pc);
}

// Product output at level l-1: out_c[i] = (u_c[i] - w_c[i]) S^-1 + d_p[i] q_l^-1 (mod q_i),
// i < l, S = q_l P: the relinearised product (d_0 + KS_0, d_1 + KS_1) divided by q_l
// with one rounding.  grid (n/TPB, l, 2B)
__global__ void k_ks_combine_rs(u64* out, size_t ps, const u64* __restrict__ u, const u64* __restrict__ w,
                                const u64* __restrict__ d, int level, int L, int alpha, ConvTables cv, int n,
                                const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = 2 * (blockIdx.x * TPB + threadIdx.x), i = blockIdx.y, c = blockIdx.z;
    const int b = c >> 1, p = c & 1;
    const u64 q = pc[i].q;
    const size_t pl = (size_t)(level + 1) * n;
    const u64* sinv = cv.mdrs + (size_t)level * cv.mdrs_stride + 2 * (alpha + 1) + (size_t)(alpha + 1) * (L + 1) + (L + 1);
    const u64* rs = cv.rescale + (size_t)level * 3 * (L + 1);
    const u64 s0 = sinv[i], s1 = sinv[(L + 1) + i], r0 = rs[i], r1 = rs[(L + 1) + i];
    const ulonglong2 uv = ld2(u + (size_t)c * (level + 1 + alpha) * n + (size_t)i * n + k);
    const ulonglong2 wv = ld2(w + (size_t)c * level * n + (size_t)i * n + k);
    const ulonglong2 dv = ld2(d + (size_t)b * 3 * pl + (size_t)p * pl + (size_t)i * n + k);
    const u64 a0 = shoup_mul(sub_mod(uv.x, wv.x, q), s0, s1, q), a1 = shoup_mul(sub_mod(uv.y, wv.y, q), s0, s1, q);
    st2(out + (size_t)c * ps + (size_t)i * n + k, add_mod(a0, shoup_mul(dv.x, r0, r1, q), q),
        add_mod(a1, shoup_mul(dv.y, r0, r1, q), q));
}

void launch_ks_combine_rs(const KernelEnv& env, u64* out, size_t ps, const u64* u, const u64* w, const u64* d, int level,
                          cudaStream_t st, int B) {
    ProfScope pf(env, KK_KS_COMBINE, st, 1, 8.0 * B * level * 8.0 * env.n, 2.0 * B * level * env.n);
    rk_launch(k_ks_combine_rs, grid2(env, level, 2 * B), TPB, 0, st, out, ps, u, w, d, level, env.L, env.alpha, env.conv, env.n,
              env.pc);
}

// ===========================================================================
// Key-switching inner product (evaluation domain), automorphism fused:
//   u_c[t][k] = sum_j ext[j][t][src(k)] * key[j][c][prime(t)][k]   (key times R)
// ===========================================================================
// Up to CH stacked ciphertexts per thread: each key word is read (or regenerated)
// once per chunk.  CH is the smallest of 1, 2, 4 that covers the stack (chunks of 4
// beyond: eight members a thread held too many registers for the occupancy that
// hides the key stream), so a single ciphertext keeps two accumulators and the digit
// loop stays unrolled.
// SEEDED: the key holds b_j only and a_j is regenerated from the key's seed.
template <int CH, bool SEEDED, bool SP>
__global__ void __launch_bounds__(TPB, (CH == 1 ? 6 : (CH == 2 ? 4 : 3))) k_ks_inner(const u64* __restrict__ ext, size_t ext_stride, const u64* __restrict__ key,
                                                  u64 seed, u64* __restrict__ u, int level, int L, int alpha, int beta, u64 galois,
                                                  int logn, int B, int accumulate, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int n = 1 << logn;
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y;
    const int b0 = blockIdx.z * CH;
    const int nb = min(CH, B - b0);
    const int pid = t <= level ? t : L + 1 + (t - level - 1);
    const PrimeConst P = pc[pid];
    const int src = galois ? galois_src(k, galois, logn) : k;
    const size_t KL = (size_t)(L + 1 + alpha) * n;
    const size_t estride = (size_t)beta * ext_stride;   // between stacked ciphertexts
    Acc128 a0[CH], a1[CH];
    const u64* kj = key + (size_t)pid * n + k;
    const u64* ej = ext + (size_t)b0 * estride + (size_t)t * n + src;
    const int T = L + 1 + alpha;
    u64 state = SEEDED ? seeded_key_state(seed, 0, T, pid, n, k) : 0;
    const u64 step = (u64)T * (u64)n * kSm64Gamma;   // one digit further in the stream
#pragma unroll 4
    for (int j = 0; j < beta; j++) {
        const u64 kb = __ldg(kj);
        const u64 ka = SEEDED ? seeded_key_word_t<SP>(state, P.q) : __ldg(kj + KL);
#pragma unroll
        for (int b = 0; b < CH; b++) {
            if (CH == 1 || b < nb) {
                const u64 e = ej[(size_t)b * estride];
                a0[b].mac(e, kb);
                a1[b].mac(e, ka);
            }
        }
        kj += (SEEDED ? 1 : 2) * KL;
        ej += ext_stride;
        state += step;
    }
    const int ul = level + 1 + alpha;
#pragma unroll
    for (int b = 0; b < CH; b++) {
        if (CH == 1 || b < nb) {
            u64* ub = u + (size_t)(b0 + b) * 2 * ul * n;
            u64 r0 = a0[b].template redc_t<SP>(P.q, P.qinv), r1 = a1[b].template redc_t<SP>(P.q, P.qinv);
            if (accumulate) {   // a further rotation's products added to the sum held in u
                r0 = add_mod(r0, ub[(size_t)t * n + k], P.q);
                r1 = add_mod(r1, ub[(size_t)ul * n + (size_t)t * n + k], P.q);
            }
            ub[(size_t)t * n + k] = r0;
            ub[(size_t)ul * n + (size_t)t * n + k] = r1;
        }
    }
}

void launch_ks_inner(const KernelEnv& env, const u64* ext, size_t ext_stride, KeyRef key, u64* u, int level, int beta,
                     u64 galois, cudaStream_t st, int B, bool accumulate) {
    // algorithmic bytes: B lifted inputs read, the key (b and a, or b alone when
    // seeded) read once per chunk, B outputs written
    const double QP = level + 1 + env.alpha;
    const int ch = B <= 1 ? 1 : B <= 2 ? 2 : 4;
    const int chunks = (B + ch - 1) / ch;
    const double key_parts = key.seeded ? 1.0 : 2.0;
    ProfScope pf(env, KK_KS_INNER, st, 1,
                 ((double)B * beta + key_parts * beta * chunks + (accumulate ? 4.0 : 2.0) * B) * QP * 8.0 * env.n,
                 2.0 * B * beta * QP * env.n);
    dim3 g(env.n / TPB, level + 1 + env.alpha, chunks);
#define RK_KSI(C, SD)                                                                                                     \
    do {                                                                                                                    \
        if (env.sp)                                                                                                         \
            rk_launch(k_ks_inner<C, SD, true>, g, TPB, 0, st, ext, ext_stride, key.data, key.seed, u, level, env.L,          \
                      env.alpha, beta, galois, env.logn, B, accumulate ? 1 : 0, env.pc);                                    \
        else                                                                                                                \
            rk_launch(k_ks_inner<C, SD, false>, g, TPB, 0, st, ext, ext_stride, key.data, key.seed, u, level, env.L,         \
                      env.alpha, beta, galois, env.logn, B, accumulate ? 1 : 0, env.pc);                                    \
    } while (0)
    if (key.seeded) {
        switch (ch) {
            case 1: RK_KSI(1, true); break;
            case 2: RK_KSI(2, true); break;
            default: RK_KSI(4, true); break;
        }
    } else {
        switch (ch) {
            case 1: RK_KSI(1, false); break;
            case 2: RK_KSI(2, false); break;
            default: RK_KSI(4, false); break;
        }
    }
#undef RK_KSI
}

// out[c][t] = base_c[t] (automorphism applied to base0 when galois0 != 0) + (u[c][t] - w[c][t]) * P^-1
// (+ addend[c][t] when addend is not null: a rotation fused with the sum x + rot(x));
// base_c points at limb 0 of one polynomial, or is null.
// z = 2b + p over B stacked ciphertexts; base_p of ciphertext b at base_p + b * bstride;
// the addend has the output's layout (polynomial c at addend + c * ps)
__global__ void k_ks_combine(u64* out, size_t ps, const u64* base0, u64 galois0, const u64* base1, size_t bstride,
                             const u64* __restrict__ u, const u64* __restrict__ w, const u64* addend, int level, int alpha,
                             ConvTables cv, int logn, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int n = 1 << logn;
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y, c = blockIdx.z;
    const int b = c >> 1, p = c & 1;
    const u64 q = pc[t].q;
    const int ul = level + 1 + alpha;
    u64 v = sub_mod(u[(size_t)c * ul * n + (size_t)t * n + k], w[(size_t)c * (level + 1) * n + (size_t)t * n + k], q);
    v = shoup_mul(v, cv.pinv[2 * t], cv.pinv[2 * t + 1], q);
    const u64* base = p == 0 ? base0 : base1;
    if (base) {
        const int src = (p == 0 && galois0) ? galois_src(k, galois0, logn) : k;
        v = add_mod(v, base[(size_t)b * bstride + (size_t)t * n + src], q);
    }
    const size_t off = (size_t)c * ps + (size_t)t * n + k;
    if (addend) v = add_mod(v, addend[off], q);
    out[off] = v;
}

void launch_ks_combine(const KernelEnv& env, u64* out, size_t ps, const u64* base0, u64 galois0, const u64* base1, size_t bstride,
                       const u64* u, const u64* w, int level, cudaStream_t st, int B, const u64* addend) {
    ProfScope pf(env, KK_KS_COMBINE, st, 1, (addend ? 9.0 : 7.0) * B * (level + 1) * 8.0 * env.n, 2.0 * B * (level + 1) * env.n);
    dim3 g(env.n / TPB, level + 1, 2 * B);
    rk_launch(k_ks_combine, g, TPB, 0, st, out, ps, base0, galois0, base1, bstride, u, w, addend, level, env.alpha, env.conv,
              env.logn, env.pc);
}

// A hoisted sum of K rotations of x (K <= 3), z = 2b + p over B stacked ciphertexts:
//   out_b.c0 = x_b.c0 + sum_k sigma_k(x_b.c0) + (u0_b - w0_b) P^-1,
//   out_b.c1 = x_b.c1 + (u1_b - w1_b) P^-1
// (x_b at x + b * bstride, poly stride ps; u the summed inner products, w ModDown's
// conversion of their P part); without `add`, x_b itself is left out.
__global__ void k_ks_combine_sum(u64* out, size_t ps, const u64* __restrict__ x, size_t bstride, GaloisSet gs, int add,
                                 const u64* __restrict__ u, const u64* __restrict__ w, int level, int alpha, ConvTables cv,
                                 int logn, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int n = 1 << logn;
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y, c = blockIdx.z;
    const int b = c >> 1, p = c & 1;
    const u64 q = pc[t].q;
    const int ul = level + 1 + alpha;
    u64 v = sub_mod(u[(size_t)c * ul * n + (size_t)t * n + k], w[(size_t)c * (level + 1) * n + (size_t)t * n + k], q);
    v = shoup_mul(v, cv.pinv[2 * t], cv.pinv[2 * t + 1], q);
    const u64* xb = x + (size_t)b * bstride + (size_t)p * ps + (size_t)t * n;
    if (p == 0)
        for (int r = 0; r < gs.K; r++) v = add_mod(v, xb[galois_src(k, gs.g[r], logn)], q);
    if (add) v = add_mod(v, xb[k], q);
    out[(size_t)b * bstride + (size_t)p * ps + (size_t)t * n + k] = v;
}

void launch_ks_combine_sum(const KernelEnv& env, u64* out, size_t ps, const u64* x, size_t bstride, const GaloisSet& gs,
                           bool add, const u64* u, const u64* w, int level, cudaStream_t st, int B) {
    ProfScope pf(env, KK_KS_COMBINE, st, 1, (7.0 + gs.K + (add ? 2.0 : 0.0)) * B * (level + 1) * 8.0 * env.n,
                 2.0 * B * (level + 1) * env.n);
    dim3 g(env.n / TPB, level + 1, 2 * B);
    rk_launch(k_ks_combine_sum, g, TPB, 0, st, out, ps, x, bstride, gs, add ? 1 : 0, u, w, level, env.alpha, env.conv,
              env.logn, env.pc);
}

// ===========================================================================
// Rescale: lift the (coefficient-domain) last limb, centred, into the lower limbs.
// last: 2 polys at stride ls; v: [2][level][n].  grid (n/TPB, level, 2)
// ===========================================================================
__global__ void k_rescale_lift(const u64* last, size_t ls, u64* v, int level, int L, ConvTables cv, int n,
                               const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = blockIdx.x * TPB + threadIdx.x, i = blockIdx.y, c = blockIdx.z;
    const u64 ql = pc[level].q;
    const u64 x = last[(size_t)c * ls + k];
    const PrimeConst P = pc[i];
    u64 r = shoup_mul(x, 1, P.one_shoup, P.q);
    if (x > (ql >> 1)) r = sub_mod(r, cv.rescale[(size_t)level * 3 * (L + 1) + 2 * (L + 1) + i], P.q);
    v[(size_t)c * level * n + (size_t)i * n + k] = r;
}

void launch_rescale_lift(const KernelEnv& env, const u64* last, size_t ls, u64* v, int level, cudaStream_t st, int polys) {
    ProfScope pf(env, KK_RESCALE, st, 1, polys * (1.0 + level) * 8.0 * env.n, 1.0 * polys * level * env.n);
    dim3 g(env.n / TPB, level, polys);
    rk_launch(k_rescale_lift, g, TPB, 0, st, last, ls, v, level, env.L, env.conv, env.n, env.pc);
}

// out[c][i] = (K_i in[c][i] - v[c][i]) * q_l^-1, i < level (K_i = 1 without SCALE;
// out may be in)
template <bool SCALE>
__global__ void k_rescale_combine(u64* out, const u64* in, size_t ps, const u64* v, int level, int L, ConvTables cv, ScalarArg K,
                                  int n, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = 2 * (blockIdx.x * TPB + threadIdx.x), i = blockIdx.y, c = blockIdx.z;
    const u64 q = pc[i].q;
    const u64* tab = cv.rescale + (size_t)level * 3 * (L + 1);
    const u64 t0 = tab[i], t1 = tab[(L + 1) + i];
    const size_t off = (size_t)c * ps + (size_t)i * n + k;
    ulonglong2 x = ld2(in + off);
    if (SCALE) {
        x.x = shoup_mul(x.x, K.w[i], K.wsh[i], q);
        x.y = shoup_mul(x.y, K.w[i], K.wsh[i], q);
    }
    const ulonglong2 vv = ld2(v + (size_t)c * level * n + (size_t)i * n + k);
    st2(out + off, shoup_mul(sub_mod(x.x, vv.x, q), t0, t1, q), shoup_mul(sub_mod(x.y, vv.y, q), t0, t1, q));
}

void launch_rescale_combine(const KernelEnv& env, u64* out, const u64* in, size_t ps, const u64* v, int level, const ScalarArg* K,
                            cudaStream_t st, int polys) {
    ProfScope pf(env, KK_RESCALE, st, 1, 3.0 * polys * level * 8.0 * env.n, 1.0 * polys * level * env.n);
    dim3 g = grid2(env, level, polys);
    if (K)
        rk_launch(k_rescale_combine<true>, g, TPB, 0, st, out, in, ps, v, level, env.L, env.conv, *K, env.n, env.pc);
    else
        rk_launch(k_rescale_combine<false>, g, TPB, 0, st, out, in, ps, v, level, env.L, env.conv, ScalarArg{}, env.n, env.pc);
}

void launch_rescale_combine(const KernelEnv& env, u64* ct, size_t ps, const u64* v, int level, cudaStream_t st, int polys) {
    launch_rescale_combine(env, ct, ct, ps, v, level, nullptr, st, polys);
}

// ===========================================================================
// Client-side helpers: signed reduction, uniform sampling, key assembly, decrypt.
// ===========================================================================
// dst[t][k] = src[k] mod prime(t) for `limbs` limbs of the LimbSet's first poly map.
__global__ void k_reduce_signed(const int64_t* src, u64* dst, LimbSet s, int n, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y, p = blockIdx.z;
    const PrimeConst P = pc[limb_prime(s, t)];
    const int64_t x = src[(size_t)p * n + k];
    const u64 ax = x < 0 ? (u64)(-(x + 1)) + 1u : (u64)x;
    u64 r = shoup_mul(ax, 1, P.one_shoup, P.q);
    if (x < 0 && r) r = P.q - r;
    dst[(size_t)p * s.poly_stride + (size_t)t * n + k] = r;
}

void launch_reduce_signed(const KernelEnv& env, const int64_t* src, const LimbSet& s, cudaStream_t st) {
    ProfScope pf(env, KK_CLIENT, st, 1, 0.0, 0.0);
    dim3 g(env.n / TPB, s.n_limbs, s.n_polys);
    rk_launch(k_reduce_signed, g, TPB, 0, st, src, s.base, s, env.n, env.pc);
}

__device__ __forceinline__ u64 splitmix64(u64 x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Uniform residues: word k of limb t of poly p from SplitMix64 of a per-word counter.
__global__ void k_uniform(LimbSet s, u64 seed, u64 stream_id, int n, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y, p = blockIdx.z;
    const u64 q = pc[limb_prime(s, t)].q;
    const u64 ctr = ((stream_id * 64 + (u64)p) * 128 + (u64)t) * (u64)n + (u64)k;
    const u64 r = splitmix64(seed ^ splitmix64(ctr));
    s.base[(size_t)p * s.poly_stride + (size_t)t * n + k] = umulhi64(r, q);
}

void launch_uniform(const KernelEnv& env, const LimbSet& s, u64 seed, u64 stream_id, cudaStream_t st) {
    ProfScope pf(env, KK_CLIENT, st, 1, 0.0, 0.0);
    dim3 g(env.n / TPB, s.n_limbs, s.n_polys);
    rk_launch(k_uniform, g, TPB, 0, st, s, seed, stream_id, env.n, env.pc);
}

// Switching-key digit in Montgomery form over all primes (eval domain):
//   b = -a s + e + gad_t s',  key_b = b R, key_a = a R.
// a, e, s' normal form; s_R = s R.  grid (n/TPB, n_primes)
__global__ void k_key_digit(u64* kb, u64* ka, const u64* a, const u64* e, const u64* s_R, const u64* sp, const u64* gad,
                            int n, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y;
    const PrimeConst P = pc[t];
    const size_t off = (size_t)t * n + k;
    const u64 as = mont_mul(a[off], s_R[off], P.q, P.qinv);
    u64 b = sub_mod(e[off], as, P.q);
    if (gad[t]) b = add_mod(b, mont_mul(sp[off], gad[t], P.q, P.qinv), P.q);   // gad stored times R
    kb[off] = mont_mul(b, P.r2, P.q, P.qinv);
    ka[off] = mont_mul(a[off], P.r2, P.q, P.qinv);
}

void launch_key_digit(const KernelEnv& env, u64* kb, u64* ka, const u64* a, const u64* e, const u64* s_R, const u64* sp,
                      const u64* gad_dev, int n_primes, cudaStream_t st) {
    ProfScope pf(env, KK_CLIENT, st, 1, 0.0, 0.0);
    dim3 g(env.n / TPB, n_primes);
    rk_launch(k_key_digit, g, TPB, 0, st, kb, ka, a, e, s_R, sp, gad_dev, env.n, env.pc);
}

// Seeded digit j of a switching key: a = (stream word) R^-1 (seeded_key_word gives the
// Montgomery form), b = e - a s + gad s' stored times R.  t over the key's primes.
__global__ void k_key_digit_seeded(u64* kb, const u64* e, const u64* s_R, const u64* sp, const u64* gad, u64 seed, int j,
                                   int T, int n, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y;
    const PrimeConst P = pc[t];
    const size_t off = (size_t)t * n + k;
    const u64 a = mont_mul(seeded_key_word(seeded_key_state(seed, j, T, t, n, k), P.q), 1, P.q, P.qinv);
    const u64 as = mont_mul(a, s_R[off], P.q, P.qinv);
    u64 b = sub_mod(e[off], as, P.q);
    if (gad[t]) b = add_mod(b, mont_mul(sp[off], gad[t], P.q, P.qinv), P.q);   // gad stored times R
    kb[off] = mont_mul(b, P.r2, P.q, P.qinv);
}

void launch_key_digit_seeded(const KernelEnv& env, u64* kb, const u64* e, const u64* s_R, const u64* sp, const u64* gad_dev,
                             u64 seed, int j, int n_primes, cudaStream_t st) {
    ProfScope pf(env, KK_CLIENT, st, 1, 0.0, 0.0);
    dim3 g(env.n / TPB, n_primes);
    rk_launch(k_key_digit_seeded, g, TPB, 0, st, kb, e, s_R, sp, gad_dev, seed, j, n_primes, env.n, env.pc);
}

// x <- x R (to Montgomery form), over `limbs` limbs of `polys` polys using LimbSet prime map
__global__ void k_to_mont(LimbSet s, int n, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y, p = blockIdx.z;
    const PrimeConst P = pc[limb_prime(s, t)];
    u64* x = s.base + (size_t)p * s.poly_stride + (size_t)t * n + k;
    *x = mont_mul(*x, P.r2, P.q, P.qinv);
}

void launch_to_mont(const KernelEnv& env, const LimbSet& s, cudaStream_t st) {
    ProfScope pf(env, KK_CLIENT, st, 1, 0.0, 0.0);
    dim3 g(env.n / TPB, s.n_limbs, s.n_polys);
    rk_launch(k_to_mont, g, TPB, 0, st, s, env.n, env.pc);
}

// out[t][k] = x[t][src(k)] (automorphism in the eval domain) over `limbs` contiguous limbs
__global__ void k_automorph(u64* out, const u64* x, u64 g, int logn) {
    RK_KERNEL_PROLOGUE();
    const int n = 1 << logn;
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y;
    out[(size_t)t * n + k] = x[(size_t)t * n + galois_src(k, g, logn)];
}

void launch_automorph(const KernelEnv& env, u64* out, const u64* x, u64 g, int limbs, cudaStream_t st) {
    ProfScope pf(env, KK_CLIENT, st, 1, 0.0, 0.0);
    dim3 g2(env.n / TPB, limbs);
    rk_launch(k_automorph, g2, TPB, 0, st, out, x, g, env.logn);
}

// m[t] = c0[t] + c1[t] s[t] (s times R), t <= level; m is [limbs][n]
__global__ void k_decrypt(u64* m, const u64* c0, const u64* c1, const u64* s_R, int n, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y;
    const PrimeConst P = pc[t];
    const size_t off = (size_t)t * n + k;
    m[off] = add_mod(c0[off], mont_mul(c1[off], s_R[off], P.q, P.qinv), P.q);
}

void launch_decrypt(const KernelEnv& env, u64* m, const u64* c0, const u64* c1, const u64* s_R, int limbs, cudaStream_t st) {
    ProfScope pf(env, KK_CLIENT, st, 1, 0.0, 0.0);
    dim3 g(env.n / TPB, limbs);
    rk_launch(k_decrypt, g, TPB, 0, st, m, c0, c1, s_R, env.n, env.pc);
}

// Public-key encryption: c0 = v pk0 + e0 + m, c1 = v pk1 + e1 (pk times R).
// r = [v | e0 | e1 | m] each [limbs][n] reduced and transformed.
__global__ void k_encrypt(u64* ct, size_t ps, const u64* r, const u64* pk, size_t pk_ps, int limbs, int n,
                          const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y;
    const PrimeConst P = pc[t];
    const size_t off = (size_t)t * n + k, pl = (size_t)limbs * n;
    const u64 v = r[off], e0 = r[pl + off], e1 = r[2 * pl + off], m = r[3 * pl + off];
    ct[off] = add_mod(add_mod(mont_mul(v, pk[off], P.q, P.qinv), e0, P.q), m, P.q);
    ct[ps + off] = add_mod(mont_mul(v, pk[pk_ps + off], P.q, P.qinv), e1, P.q);
}

void launch_encrypt(const KernelEnv& env, u64* ct, size_t ps, const u64* r, const u64* pk, size_t pk_ps, int limbs, cudaStream_t st) {
    ProfScope pf(env, KK_CLIENT, st, 1, 0.0, 0.0);
    dim3 g(env.n / TPB, limbs);
    rk_launch(k_encrypt, g, TPB, 0, st, ct, ps, r, pk, pk_ps, limbs, env.n, env.pc);
}

// pk0 = -a s + e (s times R), normal form; then both stored times R.  grid (n/TPB, limbs)
__global__ void k_pk(u64* pk, size_t ps, const u64* a, const u64* e, const u64* s_R, int n, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y;
    const PrimeConst P = pc[t];
    const size_t off = (size_t)t * n + k;
    u64 b = sub_mod(e[off], mont_mul(a[off], s_R[off], P.q, P.qinv), P.q);
    pk[off] = mont_mul(b, P.r2, P.q, P.qinv);
    pk[ps + off] = mont_mul(a[off], P.r2, P.q, P.qinv);
}

void launch_pk(const KernelEnv& env, u64* pk, size_t ps, const u64* a, const u64* e, const u64* s_R, int limbs, cudaStream_t st) {
    ProfScope pf(env, KK_CLIENT, st, 1, 0.0, 0.0);
    dim3 g(env.n / TPB, limbs);
    rk_launch(k_pk, g, TPB, 0, st, pk, ps, a, e, s_R, env.n, env.pc);
}

// s' = s * s (eval domain), inputs times R: out = s_R s_R R^-1 = s^2 R -> normal form via a second redc
__global__ void k_square_secret(u64* out, const u64* s_R, int n, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y;
    const PrimeConst P = pc[t];
    const size_t off = (size_t)t * n + k;
    const u64 sR = s_R[off];
    const u64 s = mont_redc(sR, 0, P.q, P.qinv);
    out[off] = mont_mul(s, sR, P.q, P.qinv);   // s * sR * R^-1 = s^2
}

void launch_square_secret(const KernelEnv& env, u64* out, const u64* s_R, int limbs, cudaStream_t st) {
    ProfScope pf(env, KK_CLIENT, st, 1, 0.0, 0.0);
    dim3 g(env.n / TPB, limbs);
    rk_launch(k_square_secret, g, TPB, 0, st, out, s_R, env.n, env.pc);
}

// from Montgomery form to normal form
__global__ void k_from_mont(u64* out, const u64* x, int n, const PrimeConst* __restrict__ pc) {
    RK_KERNEL_PROLOGUE();
    const int k = blockIdx.x * TPB + threadIdx.x, t = blockIdx.y;
    const PrimeConst P = pc[t];
    const size_t off = (size_t)t * n + k;
    out[off] = mont_redc(x[off], 0, P.q, P.qinv);
}

void launch_from_mont(const KernelEnv& env, u64* out, const u64* x, int limbs, cudaStream_t st) {
    ProfScope pf(env, KK_CLIENT, st, 1, 0.0, 0.0);
    dim3 g(env.n / TPB, limbs);
    rk_launch(k_from_mont, g, TPB, 0, st, out, x, env.n, env.pc);
}
