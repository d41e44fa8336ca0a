// Negacyclic NTT over 64-bit primes (sm_103a), register-blocked.
//
// n = 2^logn is split as 2^a x 2^b (a = logn/2).  The column pass runs the first a
// Cooley-Tukey stages on the 2^a-point columns {r 2^b + c}; the row pass runs the
// last b stages on the contiguous 2^b-point rows (merged psi twiddles in bit-reversed
// order, so the output index i holds the value at psi^(2 brev(i) + 1)).  The inverse
// (Gentleman-Sande) runs the row pass first and folds n^-1 into the column pass.
//
// Inside a pass a transform of T = 2^LOG points is owned by P = 2^(LOG/2) threads,
// each holding E = T/P residues in registers: the butterfly stages whose span is at
// least P run on the strided set {t + P m}, the others on the contiguous set
// {t E + m}, with one shared-memory exchange in between.  The twiddle of a
// butterfly whose lower element has in-transform index x, at span 2^v, is entry
//   (1 << (Sbase - v)) + (rho << (LOG - 1 - v)) + (x >> (v + 1))
// of the (inverse) table, Sbase = a - 1 for the column pass and logn - 1 for the row
// pass, rho the row number of a row-pass transform (0 in the column pass).
// Forward residues stay in [0, 4q) between stages, inverse ones in [0, 2q) (Shoup
// products, Harvey's lazy bounds); each transform returns [0, q).
#include <algorithm>

#include "ntt_core.cuh"

// Resident blocks of 256 threads per SM the passes are compiled for: three caps a
// thread at 80 registers, two at 128.
#ifndef RK_NTT_COL_BLOCKS
#define RK_NTT_COL_BLOCKS 3
#endif
#ifndef RK_NTT_ROW_BLOCKS
#define RK_NTT_ROW_BLOCKS 2
#endif


namespace {
using namespace nttc;

// LIFT (forward column pass only): the input is the centred lift of one limb (rescale).
template <int LOG, bool INV, bool COL, bool LIFT = false>
__global__ void __launch_bounds__(256, (LOG <= 8 ? (COL ? RK_NTT_COL_BLOCKS : RK_NTT_ROW_BLOCKS) : 2)) k_ntt_pass(LimbSet s, int logn, int loga, int units, const PrimeConst* __restrict__ pc,
                                                  const u64* __restrict__ tw) {
    RK_KERNEL_PROLOGUE();
    using S = Shape<LOG>;
    constexpr int P = S::P, E = S::E;
    extern __shared__ u64 sm[];
    const int n = 1 << logn, B = 1 << (logn - loga);
    // grid y = polynomial, z = limb: the polynomials of one limb (one prime, one twiddle
    // table) run together; the second pass of a transform walks the grid backwards, so
    // that it starts on the limbs the first pass wrote last (still in L2)
    constexpr bool REV = INV == COL;
    const int poly = REV ? gridDim.y - 1 - blockIdx.y : blockIdx.y;
    const int limb = s.limb0 + (REV ? gridDim.z - 1 - blockIdx.z : blockIdx.z);
    if (s.skip_ds && limb < s.split && limb / s.skip_ds == poly % s.skip_beta) return;   // block-uniform
    const int pid = limb_prime(s, limb);
    const PrimeConst PC = pc[pid];
    const u64 q = PC.q, q2 = 2 * q;
    u64* data = s.base + (size_t)poly * s.poly_stride + (size_t)limb * n;
    const int tid = threadIdx.x;
    int u, t, rho;
    u64* g;
    size_t gs;   // element x of this thread's transform is g[x * gs]
    if (COL) {
        u = tid % units;
        t = tid / units;
        rho = 0;
        g = data + (size_t)blockIdx.x * units + u;
        gs = (size_t)B;
    } else {
        u = tid / P;
        t = tid % P;
        rho = blockIdx.x * units + u;
        g = data + (size_t)rho * B;
        gs = 1;
    }
    const Twid tw_{tw + (size_t)pid * 2 * n, COL ? loga - 1 : logn - 1, rho};
    auto sidx = [&](int e) -> int { return COL ? e * units + u : row_slot<LOG>(u, e); };
    u64 x[E];

    if (!INV) {
        // load the strided set {t + P m}: coalesced over u (columns) or t (rows)
        if (LIFT) {
            // centred representative of the source residue x (mod lift_q), modulo q
            const u64* lg = s.lift + (size_t)poly * s.lift_stride + (size_t)blockIdx.x * units + u;
            const u64 half = s.lift_q >> 1, qlm = s.lift_mod[limb];
#pragma unroll
            for (int m = 0; m < E; m++) {
                const u64 v = lg[(size_t)(t + P * m) * gs];
                const u64 r = shoup_mul(v, 1, PC.one_shoup, q);
                x[m] = v > half ? sub_mod(r, qlm, q) : r;
            }
        } else {
#pragma unroll
            for (int m = 0; m < E; m++) x[m] = g[(size_t)(t + P * m) * gs];
        }
        fwd_strided<LOG>(x, t, tw_, q, q2);
#pragma unroll
        for (int m = 0; m < E; m++) sm[sidx(t + P * m)] = x[m];
        __syncthreads();
#pragma unroll
        for (int m = 0; m < E; m++) x[m] = sm[sidx(t * E + m)];
        fwd_contig<LOG>(x, t, tw_, q, q2);
        if (COL) {
            // column pass output stays in [0, 4q); coalesced over u
#pragma unroll
            for (int m = 0; m < E; m++) g[(size_t)(t * E + m) * gs] = x[m];
        } else {
            // each thread rewrites the slots it read, then the row leaves in the strided set
#pragma unroll
            for (int m = 0; m < E; m++) sm[sidx(t * E + m)] = x[m];
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; m++) g[t + P * m] = reduce_4q(sm[sidx(t + P * m)], q, q2);
        }
    } else {
        // load the contiguous set {t E + m}
        if (COL) {
#pragma unroll
            for (int m = 0; m < E; m++) x[m] = g[(size_t)(t * E + m) * gs];
        } else {
            const u64* gin = s.src ? s.src + (size_t)poly * s.src_stride + (size_t)limb * n + (size_t)rho * B : g;
#pragma unroll
            for (int m = 0; m < E; m++) sm[sidx(t + P * m)] = gin[t + P * m];
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; m++) x[m] = sm[sidx(t * E + m)];
            __syncthreads();
        }
        inv_contig<LOG>(x, t, tw_, q, q2);
#pragma unroll
        for (int m = 0; m < E; m++) sm[sidx(t * E + m)] = x[m];
        __syncthreads();
#pragma unroll
        for (int m = 0; m < E; m++) x[m] = sm[sidx(t + P * m)];
        inv_strided<LOG>(x, t, tw_, q, q2);
        if (COL) {   // last inverse pass: times n^-1, result in [0, q)
#pragma unroll
            for (int m = 0; m < E; m++) g[(size_t)(t + P * m) * gs] = shoup_mul(x[m], PC.ninv, PC.ninv_shoup, q);
        } else {
#pragma unroll
            for (int m = 0; m < E; m++) g[t + P * m] = x[m];
        }
    }
}


// Row pass for 256-point rows (n = 2^16 splits as 2^8 x 2^8): one warp a row, eight
// residues a thread, three register phases joined by two warp-local shared-memory
// exchanges (no block barrier):
//   set A = {t + 32 m}                 spans 128, 64, 32   (twiddles shared by the row)
//   set B = {32 (t / 4) + 4 m + t % 4} spans 16, 8, 4
//   set C = {8 t + m}                  spans 2, 1          (16-byte global accesses)
// Forward runs A, B, C and leaves from C reduced to [0, q); inverse runs C, B, A and
// leaves from A in [0, 2q).  Half the registers of the two-set form, so twice the
// resident warps.  Element x of a row sits in word x ^ ((x >> 3) & 15) of the row's
// shared buffer: every set's half-warp accesses hit 16 distinct 8-byte bank pairs.
__device__ __forceinline__ int row8_slot(int x) { return x ^ ((x >> 3) & 15); }
__device__ __forceinline__ int row8_b(int t, int m) { return ((t >> 2) << 5) | (m << 2) | (t & 3); }

template <bool INV>
__global__ void __launch_bounds__(256, 4) k_ntt_row8(LimbSet s, int logn, int loga, const PrimeConst* __restrict__ pc,
                                                   const u64* __restrict__ tw) {
    RK_KERNEL_PROLOGUE();
    extern __shared__ u64 sm[];
    const int n = 1 << logn, B = 1 << (logn - loga);
    // grid y = polynomial, z = limb; the forward row pass (a transform's second pass)
    // walks the grid backwards, starting on the limbs the column pass wrote last
    const int poly = INV ? blockIdx.y : gridDim.y - 1 - blockIdx.y;
    const int limb = s.limb0 + (INV ? blockIdx.z : gridDim.z - 1 - blockIdx.z);
    if (s.skip_ds && limb < s.split && limb / s.skip_ds == poly % s.skip_beta) return;   // block-uniform
    const int pid = limb_prime(s, limb);
    const u64 q = pc[pid].q, q2 = 2 * q;
    const int wi = threadIdx.x >> 5, t = threadIdx.x & 31;
    const int rho = blockIdx.x * (blockDim.x >> 5) + wi;
    u64* g = s.base + (size_t)poly * s.poly_stride + (size_t)limb * n + (size_t)rho * B;
    u64* row = sm + wi * 256;
    const Twid tw_{tw + (size_t)pid * 2 * n, logn - 1, rho};
    auto stage = [&](int v) { return twid_stage<8>(tw_, v); };
    u64 x[8];
    if (!INV) {
#pragma unroll
        for (int m = 0; m < 8; m++) x[m] = g[t + 32 * m];
#pragma unroll
        for (int v = 7; v >= 5; v--) {
            const int h = 1 << (v - 5);
            const ulonglong2* T = stage(v);
#pragma unroll
            for (int m = 0; m < 8; m++) {
                if (m & h) continue;
                u64 w, wsh;   // (t + 32 m) >> (v + 1) = m >> (v - 4)
                twid_fetch(T + (m >> (v - 4)), w, wsh);
                ct_bfly(x[m], x[m + h], w, wsh, q, q2);
            }
        }
#pragma unroll
        for (int m = 0; m < 8; m++) row[row8_slot(t + 32 * m)] = x[m];
        __syncwarp();
#pragma unroll
        for (int m = 0; m < 8; m++) x[m] = row[row8_slot(row8_b(t, m))];
#pragma unroll
        for (int v = 4; v >= 2; v--) {
            const int h = 1 << (v - 2);
            const ulonglong2* T = stage(v) + ((t >> 2) << (4 - v));
#pragma unroll
            for (int m = 0; m < 8; m++) {
                if (m & h) continue;
                u64 w, wsh;   // row8_b(t, m) >> (v + 1) = ((t / 4) << (4 - v)) + (4 m >> (v + 1))
                twid_fetch(T + ((m << 2) >> (v + 1)), w, wsh);
                ct_bfly(x[m], x[m + h], w, wsh, q, q2);
            }
        }
        // the slots written back were read above by this thread alone
#pragma unroll
        for (int m = 0; m < 8; m++) row[row8_slot(row8_b(t, m))] = x[m];
        __syncwarp();
#pragma unroll
        for (int m = 0; m < 8; m++) x[m] = row[row8_slot(8 * t + m)];
#pragma unroll
        for (int v = 1; v >= 0; v--) {
            const int h = 1 << v;
            const ulonglong2* T = stage(v) + ((8 * t) >> (v + 1));
#pragma unroll
            for (int m = 0; m < 8; m++) {
                if (m & h) continue;
                u64 w, wsh;
                twid_fetch(T + (m >> (v + 1)), w, wsh);
                ct_bfly(x[m], x[m + h], w, wsh, q, q2);
            }
        }
#pragma unroll
        for (int m = 0; m < 8; m += 2) {
            ulonglong2 pr;
            pr.x = reduce_4q(x[m], q, q2);
            pr.y = reduce_4q(x[m + 1], q, q2);
            reinterpret_cast<ulonglong2*>(g + 8 * t)[m >> 1] = pr;
        }
    } else {
        const u64* gin = s.src ? s.src + (size_t)poly * s.src_stride + (size_t)limb * n + (size_t)rho * B : g;
#pragma unroll
        for (int m = 0; m < 8; m += 2) {
            const ulonglong2 pr = reinterpret_cast<const ulonglong2*>(gin + 8 * t)[m >> 1];
            x[m] = pr.x;
            x[m + 1] = pr.y;
        }
#pragma unroll
        for (int v = 0; v <= 1; v++) {
            const int h = 1 << v;
            const ulonglong2* T = stage(v) + ((8 * t) >> (v + 1));
#pragma unroll
            for (int m = 0; m < 8; m++) {
                if (m & h) continue;
                u64 w, wsh;
                twid_fetch(T + (m >> (v + 1)), w, wsh);
                gs_bfly(x[m], x[m + h], w, wsh, q, q2);
            }
        }
#pragma unroll
        for (int m = 0; m < 8; m++) row[row8_slot(8 * t + m)] = x[m];
        __syncwarp();
#pragma unroll
        for (int m = 0; m < 8; m++) x[m] = row[row8_slot(row8_b(t, m))];
#pragma unroll
        for (int v = 2; v <= 4; v++) {
            const int h = 1 << (v - 2);
            const ulonglong2* T = stage(v) + ((t >> 2) << (4 - v));
#pragma unroll
            for (int m = 0; m < 8; m++) {
                if (m & h) continue;
                u64 w, wsh;
                twid_fetch(T + ((m << 2) >> (v + 1)), w, wsh);
                gs_bfly(x[m], x[m + h], w, wsh, q, q2);
            }
        }
#pragma unroll
        for (int m = 0; m < 8; m++) row[row8_slot(row8_b(t, m))] = x[m];
        __syncwarp();
#pragma unroll
        for (int m = 0; m < 8; m++) x[m] = row[row8_slot(t + 32 * m)];
#pragma unroll
        for (int v = 5; v <= 7; v++) {
            const int h = 1 << (v - 5);
            const ulonglong2* T = stage(v);
#pragma unroll
            for (int m = 0; m < 8; m++) {
                if (m & h) continue;
                u64 w, wsh;
                twid_fetch(T + (m >> (v - 4)), w, wsh);
                gs_bfly(x[m], x[m + h], w, wsh, q, q2);
            }
        }
#pragma unroll
        for (int m = 0; m < 8; m++) g[t + 32 * m] = x[m];
    }
}

// threads owning one transform of a pass
constexpr int pass_threads(int LOG, bool COL) { return (!COL && LOG == 8) ? 32 : 1 << (LOG / 2); }

// The transforms keep the general Shoup product for every prime: the cheaper product
// by a prime k 2^32 + 1 measured slower in the butterfly (its shifts and adds cost
// more issue slots than the two multiplies it saves).
template <bool INV, bool COL, bool LIFT = false>
void pass_launch(int LOG, dim3 grid, int threads, size_t smem, cudaStream_t st, const LimbSet& s, int logn, int loga,
                 int units, const PrimeConst* pc, const u64* tw) {
    if (!COL && LOG == 8) {
        rk_launch(k_ntt_row8<INV>, grid, threads, smem, st, s, logn, loga, pc, tw);
        return;
    }
    switch (LOG) {
#define RK_NTT_CASE(L)                                                                                        \
    case L:                                                                                                   \
        rk_launch(k_ntt_pass<L, INV, COL, LIFT>, grid, threads, smem, st, s, logn, loga, units, pc, tw);      \
        break;
        RK_NTT_CASE(5)
        RK_NTT_CASE(6)
        RK_NTT_CASE(7)
        RK_NTT_CASE(8)
        RK_NTT_CASE(9)
#undef RK_NTT_CASE
        default:
            throw rk_error(RK_EINVAL, "unsupported NTT pass size");
    }
}

template <bool INV, bool COL, bool LIFT = false>
void set_smem_attr() {
    const int bytes = 96 * 1024;
    cudaFuncSetAttribute(k_ntt_pass<5, INV, COL, LIFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_ntt_pass<6, INV, COL, LIFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_ntt_pass<7, INV, COL, LIFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_ntt_pass<8, INV, COL, LIFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_ntt_pass<9, INV, COL, LIFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// geometry of one pass: transforms of 2^LOG points, `count` of them per limb
struct PassGeom {
    dim3 grid;
    int threads, units;
    size_t smem;
};

bool small_set(const LimbSet& s) { return (long)s.n_limbs * s.n_polys < 16; }

// forced > 0: that many transforms a block (autotuned), clamped to the valid range
PassGeom geom(int LOG, bool COL, int count, const LimbSet& s, int sms, int forced = 0) {
    const int P = pass_threads(LOG, COL);
    int units = std::min(256 / P, count);
    const long limbs = (long)s.n_limbs * s.n_polys;
    if (forced > 0) {
        while (units > forced && units > 1) units >>= 1;
    } else {
        // small transforms (few limbs): narrower blocks until the grid covers two
        // waves, keeping two warps a block (column passes: 32-byte row segments)
        while (units > 1 && P * units > 64 && (long)(count / units) * limbs < 2L * sms) units >>= 1;
    }
    PassGeom gm;
    gm.units = units;
    gm.threads = P * units;
    gm.grid = dim3(count / units, s.n_polys, s.n_limbs);
    gm.smem = (size_t)(1 << LOG) * units * 8;
    return gm;
}

}  // namespace

void ntt_init_attributes() {
    set_smem_attr<false, false>();
    set_smem_attr<false, true>();
    set_smem_attr<false, true, true>();
    set_smem_attr<true, false>();
    set_smem_attr<true, true>();
}

namespace {

// limbs a group: all of them, or as many as keep a group within `group_bytes`
int group_limbs(const KernelEnv& env, const LimbSet& s, size_t group_bytes) {
    const size_t limb_bytes = (size_t)s.n_polys * env.n * 8;
    if (group_bytes == 0 || limb_bytes * s.n_limbs <= group_bytes) return s.n_limbs;
    const int per = (int)std::max<size_t>(1, group_bytes / limb_bytes);
    const int groups = (s.n_limbs + per - 1) / per;
    return (s.n_limbs + groups - 1) / groups;   // groups of (nearly) equal size
}

void ntt_forward_grouped(const KernelEnv& env, const LimbSet& s, cudaStream_t st, size_t group_bytes) {
    const int logn = env.logn, loga = logn / 2, logb = logn - loga;
    const int sm = small_set(s);
    const int per = group_limbs(env, s, group_bytes);
    const double limbs = (double)s.n_limbs * s.n_polys - (s.skip_ds ? (double)(s.n_polys / s.skip_beta) * s.split : 0.0);
    ProfScope ps(env, KK_NTT_FWD, st, 2 * ((s.n_limbs + per - 1) / per), 2.0 * limbs * 8.0 * env.n,
                 limbs * (env.n / 2) * env.logn);
    for (int z0 = 0; z0 < s.n_limbs; z0 += per) {
        LimbSet g = s;
        g.limb0 = s.limb0 + z0;
        g.n_limbs = std::min(per, s.n_limbs - z0);
        PassGeom c = geom(loga, true, 1 << logb, g, env.sms, env.tune ? env.tune->ntt_units[0][1][sm] : 0);
        if (g.lift)
            pass_launch<false, true, true>(loga, c.grid, c.threads, c.smem, st, g, logn, loga, c.units, env.pc, env.tw.psi);
        else
            pass_launch<false, true>(loga, c.grid, c.threads, c.smem, st, g, logn, loga, c.units, env.pc, env.tw.psi);
        PassGeom r = geom(logb, false, 1 << loga, g, env.sms, env.tune ? env.tune->ntt_units[0][0][sm] : 0);
        pass_launch<false, false>(logb, r.grid, r.threads, r.smem, st, g, logn, loga, r.units, env.pc, env.tw.psi);
    }
}

void ntt_inverse_grouped(const KernelEnv& env, const LimbSet& s, cudaStream_t st, size_t group_bytes) {
    const int logn = env.logn, loga = logn / 2, logb = logn - loga;
    const int sm = small_set(s);
    const int per = group_limbs(env, s, group_bytes);
    ProfScope ps(env, KK_NTT_INV, st, 2 * ((s.n_limbs + per - 1) / per), 2.0 * s.n_limbs * s.n_polys * 8.0 * env.n,
                 (double)s.n_limbs * s.n_polys * (env.n / 2) * env.logn);
    for (int z0 = 0; z0 < s.n_limbs; z0 += per) {
        LimbSet g = s;
        g.limb0 = s.limb0 + z0;
        g.n_limbs = std::min(per, s.n_limbs - z0);
        PassGeom r = geom(logb, false, 1 << loga, g, env.sms, env.tune ? env.tune->ntt_units[1][0][sm] : 0);
        pass_launch<true, false>(logb, r.grid, r.threads, r.smem, st, g, logn, loga, r.units, env.pc, env.tw.ipsi);
        PassGeom c = geom(loga, true, 1 << logb, g, env.sms, env.tune ? env.tune->ntt_units[1][1][sm] : 0);
        pass_launch<true, true>(loga, c.grid, c.threads, c.smem, st, g, logn, loga, c.units, env.pc, env.tw.ipsi);
    }
}

}  // namespace

void launch_ntt_forward(const KernelEnv& env, const LimbSet& s, cudaStream_t st) {
    if (s.n_limbs <= 0 || s.n_polys <= 0) return;
    ntt_forward_grouped(env, s, st, env.tune ? env.tune->ntt_group_bytes : 0);
}

void launch_ntt_inverse(const KernelEnv& env, const LimbSet& s, cudaStream_t st) {
    if (s.n_limbs <= 0 || s.n_polys <= 0) return;
    ntt_inverse_grouped(env, s, st, env.tune ? env.tune->ntt_group_bytes : 0);
}

void launch_ntt_forward_rows(const KernelEnv& env, const LimbSet& s, cudaStream_t st) {
    if (s.n_limbs <= 0 || s.n_polys <= 0) return;
    const int logn = env.logn, loga = logn / 2, logb = logn - loga;
    const double limbs = (double)s.n_limbs * s.n_polys - (s.skip_ds ? (double)(s.n_polys / s.skip_beta) * s.split : 0.0);
    ProfScope ps(env, KK_NTT_FWD, st, 1, 2.0 * limbs * 8.0 * env.n, limbs * (env.n / 2) * logb);
    PassGeom r = geom(logb, false, 1 << loga, s, env.sms, env.tune ? env.tune->ntt_units[0][0][small_set(s)] : 0);
    pass_launch<false, false>(logb, r.grid, r.threads, r.smem, st, s, logn, loga, r.units, env.pc, env.tw.psi);
}

// ---------------------------------------------------------------------------
// Autotuning of the pass block widths: every candidate width of each pass is timed
// with CUDA events on the context stream over a representative limb set (28+
// limbs for the large class, 2 x 3 limbs for the small one); the fastest is kept.
// The width changes only the launch shape, never a result.
// ---------------------------------------------------------------------------
namespace {
template <bool INV, bool COL>
float time_pass(const KernelEnv& env, const LimbSet& s, int LOG, int count, int units, cudaStream_t st, cudaEvent_t e0,
                cudaEvent_t e1, int reps) {
    const int logn = env.logn, loga = logn / 2;
    PassGeom g = geom(LOG, COL, count, s, env.sms, units);
    const u64* tw = INV ? env.tw.ipsi : env.tw.psi;
    pass_launch<INV, COL>(LOG, g.grid, g.threads, g.smem, st, s, logn, loga, g.units, env.pc, tw);   // warm
    RK_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; r++) pass_launch<INV, COL>(LOG, g.grid, g.threads, g.smem, st, s, logn, loga, g.units, env.pc, tw);
    RK_CUDA(cudaEventRecord(e1, st));
    RK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    RK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms / reps;
}
}  // namespace

// report: per [inverse][column][small] slot the chosen width and its microseconds
void ntt_autotune(rk_ctx* c, std::vector<double>& report) {
    const KernelEnv& env = c->env;
    const int logn = env.logn, loga = logn / 2, logb = logn - loga, n = env.n;
    const int L1 = c->L + 1;
    const int polys_large = std::max(1, 224 / L1);
    u64* buf = nullptr;
    RK_CUDA(rk_malloc_async((void**)&buf, (size_t)polys_large * L1 * n * 8, c->stream));
    RK_CUDA(cudaMemsetAsync(buf, 0, (size_t)polys_large * L1 * n * 8, c->stream));
    cudaEvent_t e0, e1;
    RK_CUDA(cudaEventCreate(&e0));
    RK_CUDA(cudaEventCreate(&e1));
    TuneTable t;
    try {
        for (int sm = 0; sm < 2; sm++) {
            const LimbSet s = sm ? LimbSet{buf, (size_t)L1 * n, 2, std::min(3, L1), std::min(3, L1), 0, 0}
                                 : LimbSet{buf, (size_t)L1 * n, polys_large, L1, L1, 0, 0};
            const int reps = sm ? 20 : 5;
            for (int inv = 0; inv < 2; inv++)
                for (int col = 0; col < 2; col++) {
                    const int LOG = col ? loga : logb, count = 1 << (col ? logb : loga);
                    const int P = pass_threads(LOG, col);
                    float best = 1e30f;
                    int best_u = 0;
                    for (int u = std::min(256 / P, count); u >= 1 && P * u >= 32; u >>= 1) {
                        float ms;
                        if (inv && col) ms = time_pass<true, true>(env, s, LOG, count, u, c->stream, e0, e1, reps);
                        else if (inv) ms = time_pass<true, false>(env, s, LOG, count, u, c->stream, e0, e1, reps);
                        else if (col) ms = time_pass<false, true>(env, s, LOG, count, u, c->stream, e0, e1, reps);
                        else ms = time_pass<false, false>(env, s, LOG, count, u, c->stream, e0, e1, reps);
                        if (ms < best) {
                            best = ms;
                            best_u = u;
                        }
                    }
                    t.ntt_units[inv][col][sm] = best_u;
                    report.push_back((double)best_u);
                    report.push_back(1000.0 * best);
                }
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFreeAsync(buf, c->stream);
        throw;
    }
    RK_CUDA(cudaFreeAsync(buf, c->stream));
    c->tune = t;

    // limb groups of the largest forward NTT (a top-level ModUp: every digit lifted to
    // all of Q u P): the whole set in one launch pair, or groups of at most 96, 64 or
    // 32 MiB, both passes of a group before the next
    const int beta = (L1 + c->dsize - 1) / c->dsize, T = L1 + c->alpha;
    const size_t words = (size_t)beta * T * n;
    RK_CUDA(rk_malloc_async((void**)&buf, words * 8, c->stream));
    try {
        RK_CUDA(cudaMemsetAsync(buf, 0, words * 8, c->stream));
        const LimbSet s{buf, (size_t)T * n, beta, T, T, 0, 0};
        const size_t cand[4] = {0, (size_t)96 << 20, (size_t)64 << 20, (size_t)32 << 20};
        float best = 1e30f;
        for (size_t g : cand) {
            ntt_forward_grouped(c->env, s, c->stream, g);   // warm
            RK_CUDA(cudaEventRecord(e0, c->stream));
            for (int r = 0; r < 5; r++) ntt_forward_grouped(c->env, s, c->stream, g);
            RK_CUDA(cudaEventRecord(e1, c->stream));
            RK_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            RK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            ms /= 5;
            report.push_back(1000.0 * ms);
            if (ms < best) {
                best = ms;
                c->tune.ntt_group_bytes = g;
            }
        }
        report.push_back((double)(c->tune.ntt_group_bytes >> 20));
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFreeAsync(buf, c->stream);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RK_CUDA(cudaFreeAsync(buf, c->stream));
    RK_CUDA(cudaStreamSynchronize(c->stream));
}
