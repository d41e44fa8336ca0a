// 64-bit modular arithmetic for RNS residues on sm_103a.
//
// Every prime is below 2^61, so lazy values up to 4q fit in a 64-bit word.
//  * Shoup multiplication (one operand a precomputed constant w with
//    w' = floor(w 2^64 / q)): result in [0, 2q) before the final correction.
//  * Montgomery reduction with R = 2^64 for variable x variable products and for
//    sums of products (keys and conversion constants are stored times R).
#pragma once
#include <cstdint>

typedef unsigned long long u64;
typedef unsigned __int128 u128;

#define RK_HD __host__ __device__ __forceinline__

RK_HD u64 umulhi64(u64 a, u64 b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (u64)(((u128)a * b) >> 64);
#endif
}

// a + b mod q, a, b in [0, q)
RK_HD u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}
// a - b mod q, a, b in [0, q)
RK_HD u64 sub_mod(u64 a, u64 b, u64 q) {
    return a >= b ? a - b : a + q - b;
}
// reduce x in [0, 2q) to [0, q)
RK_HD u64 reduce_2q(u64 x, u64 q) { return x >= q ? x - q : x; }

// Shoup: a * w mod q, lazily in [0, 2q); any a < 2^64.
RK_HD u64 shoup_lazy(u64 a, u64 w, u64 wp, u64 q) {
    u64 qhat = umulhi64(a, wp);
    return a * w - qhat * q;
}
RK_HD u64 shoup_mul(u64 a, u64 w, u64 wp, u64 q) { return reduce_2q(shoup_lazy(a, w, wp, q), q); }

// Montgomery reduction of T = hi 2^64 + lo with hi < q: returns T R^-1 mod q in [0, q).
// qinv = q^-1 mod 2^64.
RK_HD u64 mont_redc(u64 lo, u64 hi, u64 q, u64 qinv) {
    u64 m = lo * qinv;
    u64 mh = umulhi64(m, q);
    u64 t = hi - mh;
    return hi < mh ? t + q : t;
}

// ---------------------------------------------------------------------------
// Primes of the form q = k 2^32 + 1 (k < 2^29, so q < 2^61).  Products by q then
// need one 32-bit multiply where a general q needs three (low word) or four (high
// word):
//   x q mod 2^64          = x + ((x mod 2^32) k mod 2^32) 2^32
//   floor(m q / 2^64)     = mh k + floor((ml k + mh) / 2^32),  m = mh 2^32 + ml
//   q^-1 mod 2^64         = 1 - k 2^32            (since (1 + k 2^32)(1 - k 2^32) = 1 - k^2 2^64)
// The results are the same words as the general forms above, bit for bit.  The key-
// switching kernels take the Montgomery reductions and the seeded key word in this
// form; Shoup's product keeps the general form (with the shift and add it measured
// no faster, and slower inside the NTT butterfly).
// ---------------------------------------------------------------------------
RK_HD bool is_k32_prime(u64 q) { return (q & 0xffffffffull) == 1ull && (q >> 32) < (1ull << 29); }

RK_HD u64 mul_q_lo_k32(u64 x, u64 q) {
    return x + ((u64)((uint32_t)x * (uint32_t)(q >> 32)) << 32);
}

// floor(x q / 2^64)
RK_HD u64 mulhi_q_k32(u64 x, u64 q) {
    const uint32_t k = (uint32_t)(q >> 32);
    const u64 xh = x >> 32;
    return xh * k + (((u64)(uint32_t)x * k + xh) >> 32);
}

RK_HD u64 mont_redc_k32(u64 lo, u64 hi, u64 q) {
    const uint32_t k = (uint32_t)(q >> 32);
    const u64 m = lo - ((u64)((uint32_t)lo * k) << 32);   // lo q^-1 mod 2^64
    const u64 mh = mulhi_q_k32(m, q);
    const u64 t = hi - mh;
    return hi < mh ? t + q : t;
}

// The two forms behind one switch (SP: every prime the kernel touches is k 2^32 + 1).
template <bool SP>
RK_HD u64 shoup_lazy_t(u64 a, u64 w, u64 wp, u64 q) {
    const u64 qhat = umulhi64(a, wp);
    return a * w - (SP ? mul_q_lo_k32(qhat, q) : qhat * q);
}
template <bool SP>
RK_HD u64 shoup_mul_t(u64 a, u64 w, u64 wp, u64 q) { return reduce_2q(shoup_lazy_t<SP>(a, w, wp, q), q); }
template <bool SP>
RK_HD u64 mont_redc_t(u64 lo, u64 hi, u64 q, u64 qinv) {
    return SP ? mont_redc_k32(lo, hi, q) : mont_redc(lo, hi, q, qinv);
}
template <bool SP>
RK_HD u64 mont_mul_t(u64 a, u64 b, u64 q, u64 qinv) {
    return mont_redc_t<SP>(a * b, umulhi64(a, b), q, qinv);
}
// a * b R^-1 mod q for a < 2^64, b < q (so that hi < q)
RK_HD u64 mont_mul(u64 a, u64 b, u64 q, u64 qinv) {
    return mont_redc(a * b, umulhi64(a, b), q, qinv);
}

// 128-bit accumulator for sums of products of residues.
struct Acc128 {
    u64 lo, hi;
    RK_HD Acc128() : lo(0), hi(0) {}
    RK_HD void mac(u64 a, u64 b) {
        u64 pl = a * b, ph = umulhi64(a, b);
        lo += pl;
        hi += ph + (lo < pl);
    }
    // Reduce sum T (with T < 2q * 2^64, e.g. up to 16 products of values < 2^61
    // by values < q) to T R^-1 mod q.
    RK_HD u64 redc(u64 q, u64 qinv) const {
        u64 h = hi;
        if (h >= q) h -= q;
        return mont_redc(lo, h, q, qinv);
    }
    template <bool SP>
    RK_HD u64 redc_t(u64 q, u64 qinv) const {
        u64 h = hi;
        if (h >= q) h -= q;
        return mont_redc_t<SP>(lo, h, q, qinv);
    }
};

// Per-prime constants kept in __constant__ memory (see context.cu).
struct PrimeConst {
    u64 q;
    u64 qinv;      // q^-1 mod 2^64
    u64 r_mod;     // 2^64 mod q
    u64 r2;        // 2^128 mod q
    u64 r_shoup;   // Shoup companion of r_mod
    u64 ninv;      // n^-1 mod q
    u64 ninv_shoup;
    u64 one_shoup; // floor(2^64 / q): Shoup companion of 1 (reduces any 64-bit word)
};

#define RK_MAX_PRIMES 80
