// Rescale on caller-owned device buffers with no device allocation at all.
//
// Some callers cannot allocate device memory on the call path: for example code
// running where another runtime has already reserved the device memory in its own
// pool, or a latency-critical loop that must never enter the CUDA allocator.  This
// entry point takes the ciphertext in and out as caller-owned device buffers and
// keeps its temporary (the centred lift of the dropped residue) in a fixed array
// in device memory that the library declares at file scope, so it performs no
// cudaMalloc, cudaFree or allocating library call.
#include "kernels.cuh"

// Scratch of the allocation-free rescale: 2 * (level + 1) * n words at most.
#define RK_NOALLOC_SCRATCH_WORDS (1u << 19)   // 4 MiB
static __device__ __align__(256) u64 g_noalloc_scratch[RK_NOALLOC_SCRATCH_WORDS];

namespace {
// The array's device address, resolved by the first call on each context (with the
// context's device current) and kept in the context: a context created after the
// device was reset resolves it again, since the array may then sit elsewhere.
u64* scratch_address(rk_ctx* c) {
    if (!c->noalloc_scratch) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            throw rk_error(RK_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        c->noalloc_scratch = (u64*)p;
    }
    return c->noalloc_scratch;
}
}  // namespace

void rescale_noalloc(rk_ctx* c, const u64* in, u64* out, int l) {
    RK_REQUIRE(in && out, RK_EINVAL, "device buffers are NULL");
    RK_REQUIRE(l >= 1 && l <= c->L, RK_EINVAL, "level must be in [1, L]");
    const size_t n = c->n;
    const size_t need = (size_t)2 * (l + 1) * n;
    RK_REQUIRE(need <= RK_NOALLOC_SCRATCH_WORDS, RK_EINVAL,
               "rk_rescale_noalloc: 2*(level+1)*n = " + std::to_string(need) + " words exceeds the fixed scratch of " +
                   std::to_string(RK_NOALLOC_SCRATCH_WORDS) + " words (4 MiB)");
    const u64* in_end = in + need;
    const u64* out_end = out + (size_t)2 * l * n;
    RK_REQUIRE(out_end <= in || in_end <= out, RK_EINVAL, "input and output buffers overlap");
    RK_CUDA(cudaSetDevice(c->device));
    u64* S = scratch_address(c);
    KernelEnv env = c->env;
    env.prof = nullptr;   // never create profiling events on this path
    cudaStream_t st = c->stream;
    const size_t pin = (size_t)(l + 1) * n, pout = (size_t)l * n;
    for (int p = 0; p < 2; p++) {
        RK_CUDA(cudaMemcpyAsync(out + p * pout, in + p * pin, pout * 8, cudaMemcpyDeviceToDevice, st));
        RK_CUDA(cudaMemcpyAsync(S + p * n, in + p * pin + pout, n * 8, cudaMemcpyDeviceToDevice, st));
    }
    // every scratch word read below is written first: nothing needs clearing
    launch_ntt_inverse(env, LimbSet{S, n, 2, 1, 1, l, 0}, st);
    launch_rescale_lift(env, S, n, S + 2 * n, l, st);
    launch_ntt_forward(env, LimbSet{S + 2 * n, pout, 2, l, l, 0, 0}, st);
    launch_rescale_combine(env, out, pout, S + 2 * n, l, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw rk_error(RK_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}
