// Integer-throughput microbenchmarks of the device (the paper has no counterpart).
//
// The NTT and the basis conversions are bound by 64-bit modular arithmetic on the
// 32-bit integer multiplier, not by memory, so their roofline needs an integer peak.
// These kernels measure it with every operand in registers and no memory traffic
// beyond one word a thread: independent dependency chains per thread (instruction-
// level parallelism) over a grid that fills every SM.
//   imad      x <- x a + b, 32-bit (one multiply-add a step)
//   modmul    x <- x w mod q, Shoup's form with a precomputed companion (the NTT's)
//   butterfly the forward NTT's Cooley-Tukey butterfly on values in [0, 4q) (Harvey)
// The last two are also timed with a prime k 2^32 + 1 and the kernels' cheaper
// product by such a q.
#include <algorithm>

#include "ntt_core.cuh"

namespace {

constexpr int kChains = 8;      // independent chains a thread
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_bench_imad(uint32_t* out, int rounds, uint32_t a) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x[kChains], b[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) {
        x[i] = t + (uint32_t)i;
        b[i] = 2u * (uint32_t)i + 1u;
    }
    for (int r = 0; r < rounds; r++) {
#pragma unroll
        for (int i = 0; i < kChains; i++) x[i] = x[i] * a + b[i];
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) acc ^= x[i];
    out[t] = acc;
}

template <bool SP>
__global__ void __launch_bounds__(kThreads) k_bench_modmul(u64* out, int rounds, u64 q, u64 w, u64 wp) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    u64 x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) x[i] = (u64)t * 2654435761ull + (u64)i;
    for (int r = 0; r < rounds; r++) {
#pragma unroll
        for (int i = 0; i < kChains; i++) x[i] = shoup_lazy_t<SP>(x[i], w, wp, q);
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) acc ^= x[i];
    out[t] = acc;
}

template <bool SP>
__global__ void __launch_bounds__(kThreads) k_bench_butterfly(u64* out, int rounds, u64 q, u64 w, u64 wp) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int P = kChains / 2;   // pairs a thread
    u64 a[P], b[P];
    const u64 q2 = 2 * q;
#pragma unroll
    for (int i = 0; i < P; i++) {   // any values below 4q
        a[i] = ((u64)t * 40503ull + (u64)i) % q;
        b[i] = ((u64)t * 9176ull + 7ull * (u64)i) % q;
    }
    for (int r = 0; r < rounds; r++) {
#pragma unroll
        for (int i = 0; i < P; i++) nttc::ct_bfly<SP>(a[i], b[i], w, wp, q, q2);
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < P; i++) acc ^= a[i] + b[i];
    out[t] = acc;
}

}  // namespace

// out[0]: 32-bit multiply-adds a second, out[1]: Shoup modular products a second,
// out[2]: forward NTT butterflies a second, out[3], out[4]: the same two with the
// prime k 2^32 + 1 form (each the best of three timed launches, CUDA events on the
// context stream).  Grids of `per_sm` blocks of 256 threads on every SM, 4 and 8
// blocks tried.
void measure_alu(rk_ctx* c, double out[5]) {
    const int sms = c->env.sms;
    const size_t max_threads = (size_t)sms * 8 * kThreads;
    u64* buf = nullptr;
    RK_CUDA(rk_malloc_async((void**)&buf, max_threads * 8, c->stream));
    cudaEvent_t e0, e1;
    RK_CUDA(cudaEventCreate(&e0));
    RK_CUDA(cudaEventCreate(&e1));
    const u64 qg = c->primes[0];                   // a prime of the chain (below 2^61)
    const u64 qs = (8185ull << 32) + 1;            // a prime k 2^32 + 1 (k = 8185) near 2^45
    for (int i = 0; i < 5; i++) out[i] = 0.0;
    try {
        for (int kind = 0; kind < 5; kind++) {
            const u64 q = kind >= 3 ? qs : qg;
            const u64 w = 0x1234567ull % q, wp = (u64)(((u128)w << 64) / q);
            const int rounds = kind == 0 ? 1 << 16 : 1 << 12;
            for (int per_sm : {4, 8}) {
                const int blocks = sms * per_sm;
                const double ops = (double)blocks * kThreads * rounds * (kind == 2 || kind == 4 ? kChains / 2 : kChains);
                for (int rep = 0; rep < 4; rep++) {   // the first launch warms up
                    RK_CUDA(cudaEventRecord(e0, c->stream));
                    if (kind == 0)
                        k_bench_imad<<<blocks, kThreads, 0, c->stream>>>((uint32_t*)buf, rounds, 0x9E3779B9u);
                    else if (kind == 1)
                        k_bench_modmul<false><<<blocks, kThreads, 0, c->stream>>>(buf, rounds, q, w, wp);
                    else if (kind == 2)
                        k_bench_butterfly<false><<<blocks, kThreads, 0, c->stream>>>(buf, rounds, q, w, wp);
                    else if (kind == 3)
                        k_bench_modmul<true><<<blocks, kThreads, 0, c->stream>>>(buf, rounds, q, w, wp);
                    else
                        k_bench_butterfly<true><<<blocks, kThreads, 0, c->stream>>>(buf, rounds, q, w, wp);
                    RK_CUDA(cudaGetLastError());
                    RK_CUDA(cudaEventRecord(e1, c->stream));
                    RK_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    RK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (rep > 0 && ms > 0.f) out[kind] = std::max(out[kind], ops / (ms * 1e-3));
                }
            }
        }
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
