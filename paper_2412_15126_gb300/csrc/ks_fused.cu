// Hybrid key switching with the basis conversions fused into the NTT passes.
//
// ModUp lifts each digit of the input (coefficient domain) to the whole basis
// Q_l u P and takes it to the evaluation domain; the inner product with the
// switching key (Sec. 2, hybrid key switching) then sums digit x key over the digits.
// Four kernels carry it, none of which writes an intermediate that another pass
// re-reads in a different layout:
//   k_modup_col   conversion of digit j into limb t, then the column pass (2^a-point
//                 transforms down the columns of the 2^a x 2^b matrix).
//   k_ks_row      per output row: for every digit the row pass of that row, the
//                 automorphism as a shared-memory gather (an evaluation-domain
//                 automorphism maps each row onto one row), and the products with
//                 both key parts summed over the digits in shared memory.
//   k_moddown_col centred conversion of the P part to Q_l, then the column pass.
//   k_moddown_row the row pass, then out = base + (u - w) P^-1.
// A digit's own limbs need no lifting: k_ks_row reads them from the evaluation-
// domain input.  Every value equals the staged path's (conversion, transform and
// inner product take the same operations in the same order), bit for bit.
#include <algorithm>

#include "ntt_core.cuh"

using namespace nttc;

namespace {

// ---------------------------------------------------------------------------
// ModUp conversion of digit j into target limb tt fused with the forward column
// pass.  coef: [B][l+1][n] (coefficient domain); ext: digit j of stack member b at
// ext + (b * beta + j) * ext_stride, limb tt at + tt * n; column-pass output in [0, 4q).
// x_eval (may be null): the input in the evaluation domain (member b at
// x_eval + b * eval_stride); the blocks of a digit's own limbs then copy those limbs
// into ext (the staged path's row pass skips them).
// grid (2^b / units, limbs of the group, B * beta), block P * units
// ---------------------------------------------------------------------------
template <int LOG, bool SP>
__global__ void __launch_bounds__(256) k_modup_col(const u64* __restrict__ coef, u64* __restrict__ ext, size_t ext_stride,
                                                   const u64* __restrict__ x_eval, size_t eval_stride,
                                                   int level, int L, int alpha, int beta, int t0, ConvTables cv, int logn,
                                                   int loga, int units, const PrimeConst* __restrict__ pc,
                                                   const u64* __restrict__ tw) {
    RK_KERNEL_PROLOGUE();
    using S = Shape<LOG>;
    constexpr int P = S::P, E = S::E;
    extern __shared__ u64 sm[];
    __shared__ u64 cst[4 * RK_MAX_DIGIT];
    const int n = 1 << logn, Bw = 1 << (logn - loga);
    const int tt = t0 + blockIdx.y;
    const int j = blockIdx.z % beta, b = blockIdx.z / beta;
    const int DS = cv.dsize, lo = j * DS, hi = min(lo + DS, level + 1), ns = hi - lo;
    if (tt >= lo && tt < hi) {   // block-uniform: the digit's own limb
        if (x_eval) {
            const int u = threadIdx.x % units, t = threadIdx.x / units, col = blockIdx.x * units + u;
            const u64* src = x_eval + (size_t)b * eval_stride + (size_t)tt * n + col;
            u64* dst = ext + ((size_t)b * beta + j) * ext_stride + (size_t)tt * n + col;
#pragma unroll
            for (int m = 0; m < E; m++) dst[(size_t)(t + P * m) * Bw] = src[(size_t)(t + P * m) * Bw];
        }
        return;
    }
    const int pid = tt <= level ? tt : L + 1 + (tt - level - 1);
    const PrimeConst PC = pc[pid];
    const u64 q = PC.q, q2 = 2 * q;
    const u64* tab = cv.modup + ((size_t)level * cv.beta_max + j) * cv.modup_stride;
    const int Trow = L + 1 + alpha;
    if (threadIdx.x < ns) {
        const int i = threadIdx.x;
        cst[i] = tab[i];                                   // (D/q_i)^-1 mod q_i
        cst[RK_MAX_DIGIT + i] = tab[DS + i];               // its Shoup companion
        cst[2 * RK_MAX_DIGIT + i] = pc[lo + i].q;
        cst[3 * RK_MAX_DIGIT + i] = tab[2 * DS + (size_t)i * Trow + tt];   // (D/q_i) R mod prime(tt)
    }
    __syncthreads();
    const u64* xb = coef + ((size_t)b * (level + 1) + lo) * n;
    const int tid = threadIdx.x, u = tid % units, t = tid / units;
    const int col = blockIdx.x * units + u;
    u64 x[E];
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int idx = (t + P * m) * Bw + col;
        Acc128 acc;
#pragma unroll
        for (int i = 0; i < RK_MAX_DIGIT; i++) {
            if (i < ns) {
                const u64 y = shoup_mul(xb[(size_t)i * n + idx], cst[i], cst[RK_MAX_DIGIT + i], cst[2 * RK_MAX_DIGIT + i]);
                acc.mac(y, cst[3 * RK_MAX_DIGIT + i]);
            }
        }
        x[m] = acc.template redc_t<SP>(q, PC.qinv);
    }
    const Twid tw_{tw + (size_t)pid * 2 * n, loga - 1, 0};
    fwd_strided<LOG>(x, t, tw_, q, q2);
#pragma unroll
    for (int m = 0; m < E; m++) sm[(t + P * m) * units + u] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; m++) x[m] = sm[(t * E + m) * units + u];
    fwd_contig<LOG>(x, t, tw_, q, q2);
    u64* out = ext + ((size_t)b * beta + j) * ext_stride + (size_t)tt * n + col;
#pragma unroll
    for (int m = 0; m < E; m++) out[(size_t)(t * E + m) * Bw] = x[m];
}

// ---------------------------------------------------------------------------
// Row pass + inner product.  For output row rr of limb tt (stack member b):
//   u_c[tt][k] = sum_j ext_j[tt][src(k)] * key_j,c[tt][k] R^-1,  c = 0, 1
// src the automorphism's source index (identity when galois = 0); ext_j holds the
// column-pass output, except the digit's own limbs, read from the evaluation-domain
// input x_eval + b * eval_stride.  u: [B][2][l+1+alpha][n].
// grid (2^a / units, limbs of the group, B), block P * units
// ---------------------------------------------------------------------------
template <int LOG>
__global__ void __launch_bounds__(2048 / Shape<LOG>::E, (LOG >= 7 ? 3 : 2)) k_ks_row(const u64* __restrict__ ext, size_t ext_stride, const u64* __restrict__ x_eval,
                                                size_t eval_stride, const u64* __restrict__ key, u64 seed, int seeded,
                                                u64* __restrict__ uo, int level,
                                                int L, int alpha, int beta, int dsize, int t0, u64 galois, int logn, int units,
                                                const PrimeConst* __restrict__ pc, const u64* __restrict__ tw) {
    RK_KERNEL_PROLOGUE();
    using S = Shape<LOG>;
    constexpr int P = S::P, E = S::E, T = S::T;
    extern __shared__ u64 sm[];
    const int n = 1 << logn, logb = LOG;
    const int tt = t0 + blockIdx.y, b = blockIdx.z;
    const int pid = tt <= level ? tt : L + 1 + (tt - level - 1);
    const PrimeConst PC = pc[pid];
    const u64 q = PC.q, q2 = 2 * q;
    const int tid = threadIdx.x, u = tid / P, t = tid % P;
    const int rr = blockIdx.x * units + u;                                                  // output row
    const int rho = galois ? (galois_src(rr << logb, galois, logn) >> logb) : rr;          // its source row
    // shared memory: row buffers [units][T], the two sums [2][units][T], and the slot
    // of the source of each output element t + P m ([m][tid], u16)
    u64* acc = sm + (size_t)units * T;
    unsigned short* spos = reinterpret_cast<unsigned short*>(sm + (size_t)3 * units * T);
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int xo = t + P * m;
        const int xs = galois ? (galois_src((rr << logb) + xo, galois, logn) & (T - 1)) : xo;
        spos[m * blockDim.x + tid] = (unsigned short)row_slot<LOG>(0, xs);
        acc[(size_t)u * T + xo] = 0;
        acc[(size_t)(units + u) * T + xo] = 0;
    }
    const Twid tw_{tw + (size_t)pid * 2 * n, logn - 1, rho};
    const size_t KL = (size_t)(L + 1 + alpha) * n;
    const u64* krow = key + (size_t)pid * n + ((size_t)rr << logb);
    const u64* erow = ext + (size_t)b * beta * ext_stride + (size_t)tt * n + ((size_t)rho << logb);
    const u64* srow = sm + (size_t)u * T;
    u64* a0 = acc + (size_t)u * T;
    u64* a1 = acc + (size_t)(units + u) * T;
    u64 x[E];
    const int own = tt <= level ? tt / dsize : -1;
    for (int j = 0; j < beta; j++) {
        if (j == own) {   // block-uniform: this limb of the digit is the input itself
            const u64* xr = x_eval + (size_t)b * eval_stride + (size_t)tt * n + ((size_t)rho << logb);
#pragma unroll
            for (int m = 0; m < E; m++) sm[row_slot<LOG>(u, t + P * m)] = xr[t + P * m];
        } else {
            const u64* xr = erow + (size_t)j * ext_stride;
#pragma unroll
            for (int m = 0; m < E; m++) x[m] = xr[t + P * m];
            fwd_strided<LOG>(x, t, tw_, q, q2);
#pragma unroll
            for (int m = 0; m < E; m++) sm[row_slot<LOG>(u, t + P * m)] = x[m];
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; m++) x[m] = sm[row_slot<LOG>(u, t * E + m)];
            fwd_contig<LOG>(x, t, tw_, q, q2);
#pragma unroll
            for (int m = 0; m < E; m++) sm[row_slot<LOG>(u, t * E + m)] = reduce_4q(x[m], q, q2);
        }
        __syncthreads();
        const u64* kb = krow + (size_t)j * (seeded ? 1 : 2) * KL;
#pragma unroll 4
        for (int m = 0; m < E; m++) {
            const int xo = t + P * m;
            const u64 e = srow[spos[m * blockDim.x + tid]];
            const u64 ka = seeded ? seeded_key_word(seeded_key_state(seed, j, L + 1 + alpha, pid, n, (rr << logb) + xo), q)
                                  : __ldg(kb + KL + xo);
            a0[xo] = add_mod(a0[xo], mont_mul(e, __ldg(kb + xo), q, PC.qinv), q);
            a1[xo] = add_mod(a1[xo], mont_mul(e, ka, q, PC.qinv), q);
        }
        __syncthreads();
    }
    const int QP = level + 1 + alpha;
    u64* o = uo + (size_t)b * 2 * QP * n + (size_t)tt * n + ((size_t)rr << logb);
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int xo = t + P * m;
        o[xo] = a0[xo];
        o[(size_t)QP * n + xo] = a1[xo];
    }
}

// ---------------------------------------------------------------------------
// ModDown: centred conversion of the P part of u (coefficient domain) into limb i
// of Q_l, fused with the forward column pass.  u: [polys][l+1+alpha][n];
// w: [polys][l+1][n] column-pass output.  grid (2^b / units, l+1, polys)
// ---------------------------------------------------------------------------
template <int LOG>
__global__ void __launch_bounds__(256) k_moddown_col(const u64* __restrict__ uin, u64* __restrict__ w, int level, int L,
                                                     int alpha, ConvTables cv, int logn, int loga, int units,
                                                     const PrimeConst* __restrict__ pc, const u64* __restrict__ tw) {
    RK_KERNEL_PROLOGUE();
    using S = Shape<LOG>;
    constexpr int P = S::P, E = S::E;
    extern __shared__ u64 sm[];
    __shared__ u64 cst[4 * RK_MAX_SPECIAL];
    const int n = 1 << logn, Bw = 1 << (logn - loga);
    const int i = blockIdx.y, c = blockIdx.z;
    const int ul = level + 1 + alpha;
    const PrimeConst PC = pc[i];
    const u64 q = PC.q, q2 = 2 * q;
    const u64* cm = cv.moddown + 2 * alpha;
    if (threadIdx.x < alpha) {
        const int kk = threadIdx.x;
        cst[kk] = cv.moddown[kk];                              // (P/p_k)^-1 mod p_k
        cst[RK_MAX_SPECIAL + kk] = cv.moddown[alpha + kk];     // its Shoup companion
        cst[2 * RK_MAX_SPECIAL + kk] = pc[L + 1 + kk].q;
        cst[3 * RK_MAX_SPECIAL + kk] = cm[(size_t)kk * (L + 1) + i];   // (P/p_k) R mod q_i
    }
    __syncthreads();
    const u64 pm = cm[(size_t)alpha * (L + 1) + i];            // P mod q_i
    const u64* up = uin + (size_t)c * ul * n + (size_t)(level + 1) * n;
    const int tid = threadIdx.x, u = tid % units, t = tid / units;
    const int col = blockIdx.x * units + u;
    u64 x[E];
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int idx = (t + P * m) * Bw + col;
        Acc128 acc;
        int nneg = 0;
#pragma unroll
        for (int kk = 0; kk < RK_MAX_SPECIAL; kk++) {
            if (kk < alpha) {
                const u64 pk = cst[2 * RK_MAX_SPECIAL + kk];
                const u64 y = shoup_mul(up[(size_t)kk * n + idx], cst[kk], cst[RK_MAX_SPECIAL + kk], pk);
                nneg += y > (pk >> 1) ? 1 : 0;   // centred term: y (P/p_k) - P
                acc.mac(y, cst[3 * RK_MAX_SPECIAL + kk]);
            }
        }
        u64 r = acc.redc(q, PC.qinv);
        for (int z = 0; z < nneg; z++) r = sub_mod(r, pm, q);
        x[m] = r;
    }
    const Twid tw_{tw + (size_t)i * 2 * n, loga - 1, 0};
    fwd_strided<LOG>(x, t, tw_, q, q2);
#pragma unroll
    for (int m = 0; m < E; m++) sm[(t + P * m) * units + u] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; m++) x[m] = sm[(t * E + m) * units + u];
    fwd_contig<LOG>(x, t, tw_, q, q2);
    u64* out = w + ((size_t)c * (level + 1) + i) * n + col;
#pragma unroll
    for (int m = 0; m < E; m++) out[(size_t)(t * E + m) * Bw] = x[m];
}

// ---------------------------------------------------------------------------
// ModDown row pass + combine: w's row pass, then for z = 2b + p
//   out[z][i][k] = base_p[b][i][src(k)] + (u[z][i][k] - w[z][i][k]) P^-1
// (automorphism galois0 on base0 only; a null base adds nothing).
// grid (2^a / units, l+1, 2B), block P * units
// ---------------------------------------------------------------------------
template <int LOG>
__global__ void __launch_bounds__(256) k_moddown_row(u64* __restrict__ out, size_t ps, const u64* base0, u64 galois0,
                                                     const u64* base1, size_t bstride, const u64* __restrict__ uin,
                                                     const u64* __restrict__ w, int level, int alpha, ConvTables cv, int logn,
                                                     int units, const PrimeConst* __restrict__ pc,
                                                     const u64* __restrict__ tw) {
    RK_KERNEL_PROLOGUE();
    using S = Shape<LOG>;
    constexpr int P = S::P, E = S::E;
    extern __shared__ u64 sm[];
    const int n = 1 << logn, logb = LOG;
    const int i = blockIdx.y, z = blockIdx.z, b = z >> 1, p = z & 1;
    const PrimeConst PC = pc[i];
    const u64 q = PC.q, q2 = 2 * q;
    const int tid = threadIdx.x, u = tid / P, t = tid % P;
    const int rho = blockIdx.x * units + u;
    const size_t row0 = (size_t)rho << logb;
    const u64* wr = w + ((size_t)z * (level + 1) + i) * n + row0;
    u64 x[E];
#pragma unroll
    for (int m = 0; m < E; m++) x[m] = wr[t + P * m];
    const Twid tw_{tw + (size_t)i * 2 * n, logn - 1, rho};
    fwd_strided<LOG>(x, t, tw_, q, q2);
#pragma unroll
    for (int m = 0; m < E; m++) sm[row_slot<LOG>(u, t + P * m)] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; m++) x[m] = sm[row_slot<LOG>(u, t * E + m)];
    fwd_contig<LOG>(x, t, tw_, q, q2);
#pragma unroll
    for (int m = 0; m < E; m++) sm[row_slot<LOG>(u, t * E + m)] = x[m];
    __syncthreads();
    const int ul = level + 1 + alpha;
    const u64* ur = uin + ((size_t)z * ul + i) * n + row0;
    const u64* base = p == 0 ? base0 : base1;
    const u64 pinv = cv.pinv[2 * i], pinv_sh = cv.pinv[2 * i + 1];
    u64* o = out + (size_t)z * ps + (size_t)i * n + row0;
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int xo = t + P * m;
        const u64 wv = reduce_4q(sm[row_slot<LOG>(u, xo)], q, q2);
        u64 v = sub_mod(ur[xo], wv, q);
        v = shoup_mul(v, pinv, pinv_sh, q);
        if (base) {
            const int src = (p == 0 && galois0) ? galois_src((int)row0 + xo, galois0, logn) : (int)row0 + xo;
            v = add_mod(v, base[(size_t)b * bstride + (size_t)i * n + src], q);
        }
        o[xo] = v;
    }
}

// geometry: transforms of 2^LOG points, `count` of them per limb, up to 256 threads
struct Geom {
    int units, threads, blocks;
};
Geom geom_of(int LOG, int count) {
    const int P = 1 << (LOG / 2);
    Geom g;
    g.units = std::min(256 / P, count);
    g.threads = P * g.units;
    g.blocks = count / g.units;
    return g;
}

}  // namespace

#define RK_LOG_SWITCH(LOG, CALL)                                                         \
    switch (LOG) {                                                                       \
        case 5: { constexpr int LG = 5; CALL; } break;                                   \
        case 6: { constexpr int LG = 6; CALL; } break;                                   \
        case 7: { constexpr int LG = 7; CALL; } break;                                   \
        case 8: { constexpr int LG = 8; CALL; } break;                                   \
        case 9: { constexpr int LG = 9; CALL; } break;                                   \
        default: throw rk_error(RK_EINVAL, "unsupported NTT pass size");                 \
    }

void ks_fused_init_attributes() {
    const int bytes = 96 * 1024;
#define RK_ATTR(LG)                                                                                        \
    cudaFuncSetAttribute(k_modup_col<LG, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);      \
    cudaFuncSetAttribute(k_modup_col<LG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);       \
    cudaFuncSetAttribute(k_ks_row<LG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * bytes);            \
    cudaFuncSetAttribute(k_moddown_col<LG>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);           \
    cudaFuncSetAttribute(k_moddown_row<LG>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    RK_ATTR(5) RK_ATTR(6) RK_ATTR(7) RK_ATTR(8) RK_ATTR(9)
#undef RK_ATTR
}

void launch_modup_col(const KernelEnv& env, const u64* coef, u64* ext, size_t ext_stride, int level, int beta, int t0, int limbs,
                      cudaStream_t st, int B, const u64* x_eval, size_t eval_stride) {
    if (limbs <= 0) return;
    const int logn = env.logn, loga = logn / 2, logb = logn - loga;
    // algorithmic bytes: the digits read once, every lifted limb of the group written
    const int own = std::max(0, std::min(t0 + limbs, level + 1) - t0);
    ProfScope pf(env, KK_MODUP, st, 1, B * ((double)(level + 1) * limbs / (level + 1 + env.alpha) + (double)beta * limbs - own) * 8.0 * env.n,
                 (double)B * limbs * (level + 1) * env.n);
    const Geom g = geom_of(loga, 1 << logb);
    const dim3 grid(g.blocks, limbs, B * beta);
    const size_t smem = (size_t)(1 << loga) * g.units * 8;
    if (env.sp)
        RK_LOG_SWITCH(loga, (rk_launch(k_modup_col<LG, true>, grid, g.threads, smem, st, coef, ext, ext_stride, x_eval,
                                       eval_stride, level, env.L, env.alpha, beta, t0, env.conv, logn, loga, g.units, env.pc,
                                       env.tw.psi)))
    else
        RK_LOG_SWITCH(loga, (rk_launch(k_modup_col<LG, false>, grid, g.threads, smem, st, coef, ext, ext_stride, x_eval,
                                       eval_stride, level, env.L, env.alpha, beta, t0, env.conv, logn, loga, g.units, env.pc,
                                       env.tw.psi)))
}

void launch_ks_row(const KernelEnv& env, const u64* ext, size_t ext_stride, const u64* x_eval, size_t eval_stride, KeyRef key,
                   u64* u, int level, int beta, int t0, int limbs, u64 galois, cudaStream_t st, int B) {
    if (limbs <= 0) return;
    const int logn = env.logn, loga = logn / 2, logb = logn - loga;
    // algorithmic bytes: each digit's limb read once, the key read once, u written
    ProfScope pf(env, KK_KS_INNER, st, 1, ((double)B * beta + (key.seeded ? 1.0 : 2.0) * beta + 2.0 * B) * limbs * 8.0 * env.n,
                 2.0 * B * beta * limbs * env.n);
    // 2048 elements a block (26 bytes of shared memory each): four blocks an SM
    const int P = 1 << (logb / 2);
    Geom g;
    g.units = std::min(std::max(1, 2048 >> logb), 1 << loga);
    g.threads = P * g.units;
    g.blocks = (1 << loga) / g.units;
    const dim3 grid(g.blocks, limbs, B);
    const size_t smem = (size_t)(1 << logb) * g.units * 26;
    RK_LOG_SWITCH(logb, (rk_launch(k_ks_row<LG>, grid, g.threads, smem, st, ext, ext_stride, x_eval, eval_stride, key.data, key.seed,
                                                                     key.seeded, u, level, env.L,
                                                                     env.alpha, beta, env.conv.dsize, t0, galois, logn, g.units,
                                                                     env.pc, env.tw.psi)));
}

void launch_moddown_col(const KernelEnv& env, const u64* u, u64* w, int level, cudaStream_t st, int polys) {
    const int logn = env.logn, loga = logn / 2, logb = logn - loga;
    ProfScope pf(env, KK_MODDOWN, st, 1, polys * (1.0 * env.alpha + (level + 1)) * 8.0 * env.n,
                 1.0 * polys * (level + 1) * env.alpha * env.n);
    const Geom g = geom_of(loga, 1 << logb);
    const dim3 grid(g.blocks, level + 1, polys);
    const size_t smem = (size_t)(1 << loga) * g.units * 8;
    RK_LOG_SWITCH(loga, (rk_launch(k_moddown_col<LG>, grid, g.threads, smem, st, u, w, level, env.L, env.alpha, env.conv, logn, loga,
                                                                          g.units, env.pc, env.tw.psi)));
}

void launch_moddown_row(const KernelEnv& env, u64* out, size_t ps, const u64* base0, u64 galois0, const u64* base1, size_t bstride,
                        const u64* u, const u64* w, int level, cudaStream_t st, int B) {
    const int logn = env.logn, loga = logn / 2, logb = logn - loga;
    ProfScope pf(env, KK_KS_COMBINE, st, 1, 7.0 * B * (level + 1) * 8.0 * env.n, 2.0 * B * (level + 1) * env.n);
    const Geom g = geom_of(logb, 1 << loga);
    const dim3 grid(g.blocks, level + 1, 2 * B);
    const size_t smem = (size_t)(1 << logb) * g.units * 8;
    RK_LOG_SWITCH(logb, (rk_launch(k_moddown_row<LG>, grid, g.threads, smem, st, out, ps, base0, galois0, base1, bstride, u, w, level,
                                                                          env.alpha, env.conv, logn, g.units, env.pc, env.tw.psi)));
}
