// Building blocks of the register-blocked negacyclic NTT (sm_103a).
//
// A transform of T = 2^LOG points is owned by P = 2^(LOG/2) threads, each holding
// E = T/P residues in registers.  Butterfly stages whose span is at least P run on
// the strided set x[m] = element (t + P m) of thread t, the others on the contiguous
// set x[m] = element (t E + m); a pass moves between the two sets with one
// shared-memory exchange.  The twiddle of a butterfly whose lower element has
// in-transform index x, at span 2^v, is entry
//   (1 << (Sbase - v)) + (rho << (LOG - 1 - v)) + (x >> (v + 1))
// of the (inverse) table: Sbase = a - 1 and rho = 0 for the 2^a-point column pass,
// Sbase = logn - 1 and rho = the row number for the 2^b-point row pass.  Forward
// residues stay in [0, 4q) between stages (Harvey), inverse ones in [0, 2q).
#pragma once
#include "kernels.cuh"

namespace nttc {

// Cooley-Tukey butterfly on values in [0, 4q): one conditional subtraction.  SP: q is
// a prime k 2^32 + 1 (cheaper product by q, same result).
template <bool SP = false>
__device__ __forceinline__ void ct_bfly(u64& a, u64& b, u64 w, u64 wsh, u64 q, u64 q2) {
    u64 U = a;
    if (U >= q2) U -= q2;
    const u64 V = shoup_lazy_t<SP>(b, w, wsh, q);   // [0, 2q) for any 64-bit input
    a = U + V;
    b = U + q2 - V;
}

__device__ __forceinline__ u64 reduce_4q(u64 x, u64 q, u64 q2) {
    if (x >= q2) x -= q2;
    return x >= q ? x - q : x;
}

// Gentleman-Sande butterfly on values in [0, 2q).
template <bool SP = false>
__device__ __forceinline__ void gs_bfly(u64& a, u64& b, u64 w, u64 wsh, u64 q, u64 q2) {
    u64 U = a, V = b;
    u64 x = U + V;
    if (x >= q2) x -= q2;
    a = x;
    b = shoup_lazy_t<SP>(U + q2 - V, w, wsh, q);
}

template <int LOG>
struct Shape {
    static constexpr int T = 1 << LOG, LOGP = LOG / 2, P = 1 << LOGP, LOGE = LOG - LOGP, E = 1 << LOGE;
};

// twiddle table of one prime ((w, Shoup companion) pairs) and the position of the
// transform in the pass
struct Twid {
    const u64* W;
    int Sbase, rho;
};

// First (w, Shoup) pair of stage v of the transform (g = 0); a stage's loads then
// differ from it by offsets the unrolled loops know at compile time.
template <int LOG>
__device__ __forceinline__ const ulonglong2* twid_stage(const Twid& tw, int v) {
    return reinterpret_cast<const ulonglong2*>(tw.W) + (1 << (tw.Sbase - v)) + (tw.rho << (LOG - 1 - v));
}

__device__ __forceinline__ void twid_fetch(const ulonglong2* p, u64& w, u64& wsh) {
    const ulonglong2 pr = __ldg(p);
    w = pr.x;
    wsh = pr.y;
}

// forward stages with span 2^v >= P (v = LOG-1 .. LOGP) on the strided set
template <int LOG, bool SP = false>
__device__ __forceinline__ void fwd_strided(u64 (&x)[Shape<LOG>::E], int t, const Twid& tw, u64 q, u64 q2) {
    using S = Shape<LOG>;
#pragma unroll
    for (int v = LOG - 1; v >= S::LOGP; v--) {
        const int h = 1 << (v - S::LOGP);
        const ulonglong2* T = twid_stage<LOG>(tw, v);
#pragma unroll
        for (int m = 0; m < S::E; m++) {
            if (m & h) continue;
            u64 w, wsh;   // (t + P m) >> (v + 1) = m >> (v + 1 - LOGP): shared by the whole transform
            twid_fetch(T + (m >> (v + 1 - S::LOGP)), w, wsh);
            ct_bfly<SP>(x[m], x[m + h], w, wsh, q, q2);
        }
    }
}

// forward stages with span 2^v < P (v = LOGP-1 .. 0) on the contiguous set
template <int LOG, bool SP = false>
__device__ __forceinline__ void fwd_contig(u64 (&x)[Shape<LOG>::E], int t, const Twid& tw, u64 q, u64 q2) {
    using S = Shape<LOG>;
#pragma unroll
    for (int v = S::LOGP - 1; v >= 0; v--) {
        const int h = 1 << v;
        const ulonglong2* T = twid_stage<LOG>(tw, v) + (t << (S::LOGE - v - 1));
#pragma unroll
        for (int m = 0; m < S::E; m++) {
            if (m & h) continue;
            u64 w, wsh;   // (t E + m) >> (v + 1) = t E / 2^(v+1) + (m >> (v + 1))
            twid_fetch(T + (m >> (v + 1)), w, wsh);
            ct_bfly<SP>(x[m], x[m + h], w, wsh, q, q2);
        }
    }
}

// inverse stages with span 2^v < P (v = 0 .. LOGP-1) on the contiguous set
template <int LOG, bool SP = false>
__device__ __forceinline__ void inv_contig(u64 (&x)[Shape<LOG>::E], int t, const Twid& tw, u64 q, u64 q2) {
    using S = Shape<LOG>;
#pragma unroll
    for (int v = 0; v < S::LOGP; v++) {
        const int h = 1 << v;
        const ulonglong2* T = twid_stage<LOG>(tw, v) + (t << (S::LOGE - v - 1));
#pragma unroll
        for (int m = 0; m < S::E; m++) {
            if (m & h) continue;
            u64 w, wsh;
            twid_fetch(T + (m >> (v + 1)), w, wsh);
            gs_bfly<SP>(x[m], x[m + h], w, wsh, q, q2);
        }
    }
}

// inverse stages with span 2^v >= P (v = LOGP .. LOG-1) on the strided set
template <int LOG, bool SP = false>
__device__ __forceinline__ void inv_strided(u64 (&x)[Shape<LOG>::E], int t, const Twid& tw, u64 q, u64 q2) {
    using S = Shape<LOG>;
#pragma unroll
    for (int v = S::LOGP; v < LOG; v++) {
        const int h = 1 << (v - S::LOGP);
        const ulonglong2* T = twid_stage<LOG>(tw, v);
#pragma unroll
        for (int m = 0; m < S::E; m++) {
            if (m & h) continue;
            u64 w, wsh;
            twid_fetch(T + (m >> (v + 1 - S::LOGP)), w, wsh);
            gs_bfly<SP>(x[m], x[m + h], w, wsh, q, q2);
        }
    }
}

// shared-memory slot of element e of row u in a row pass: rows are swizzled so that
// the strided and the contiguous access patterns both avoid bank conflicts
template <int LOG>
__device__ __forceinline__ int row_slot(int u, int e) {
    using S = Shape<LOG>;
    return u * S::T + (e ^ ((e >> S::LOGE) & (S::E - 1)));
}

}  // namespace nttc

__device__ __forceinline__ int brev_bits(unsigned x, int bits) { return (int)(__brev(x) >> (32 - bits)); }

// Automorphism X -> X^g in the evaluation domain: output index k takes the input
// at galois_src(k) (index i holds the value at psi^(2 brev(i) + 1)).
__device__ __forceinline__ int galois_src(int k, u64 g, int logn) {
    unsigned two_n_mask = (2u << logn) - 1u;
    unsigned e = 2u * (unsigned)brev_bits((unsigned)k, logn) + 1u;
    unsigned e2 = (unsigned)((e * (unsigned)g) & two_n_mask);
    return brev_bits((e2 - 1u) >> 1, logn);
}
