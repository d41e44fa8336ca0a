// Launchers of the CUDA kernels (kernels.cu).  All take a KernelEnv with the
// device tables and enqueue on the given stream; none allocates.
#pragma once
#include "rk_internal.cuh"

// Programmatic dependent launch: every kernel is launched so that it may begin while
// its predecessor on the stream finishes.  Each kernel lets its own successor begin
// launching at once and then waits for its predecessor's completion (and memory)
// before touching any global memory, so stream order is kept for every access;
// only the launch latency overlaps.  RK_PDL=0 builds plain launches.
#ifndef RK_PDL
#define RK_PDL 1
#endif
#if RK_PDL
#define RK_KERNEL_PROLOGUE() asm volatile("griddepcontrol.launch_dependents;\n\tgriddepcontrol.wait;" ::: "memory")
#else
#define RK_KERNEL_PROLOGUE() ((void)0)
#endif

template <typename... KArgs, typename... Args>
inline void rk_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
#if RK_PDL
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    if (e != cudaSuccess) throw rk_error(RK_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
#else
    kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
#endif
}


// Counts every launch; when `kind` is among the profiled kinds, brackets the launch(es)
// with CUDA events on the launching stream and accumulates the algorithmic bytes/products.
struct ProfScope {
    Profiler* p;
    bool on = false;
    int kind;
    cudaStream_t st;
    double bytes, ops;
    ProfScope(const KernelEnv& e, int k, cudaStream_t s, int nlaunch, double b, double o)
        : p(e.prof), kind(k), st(s), bytes(b), ops(o) {
        if (!p) return;
        p->launches += (uint64_t)nlaunch;
        if ((p->mask & (1u << kind)) && !p->paused) {
            on = true;
            record();
        }
    }
    void record() {
        if (p->used == p->ev.size()) {
            cudaEvent_t ev;
            cudaEventCreate(&ev);
            p->ev.push_back(ev);
            p->ev_kind.push_back(-1);
        }
        p->ev_kind[p->used] = kind;
        cudaEventRecord(p->ev[p->used++], st);
    }
    ~ProfScope() {
        if (on) {
            record();
            p->bytes[kind] += bytes;
            p->ops[kind] += ops;
            p->timed[kind]++;
        }
    }
};

void ntt_init_attributes();
void launch_ntt_forward(const KernelEnv& env, const LimbSet& s, cudaStream_t st);
void launch_ntt_inverse(const KernelEnv& env, const LimbSet& s, cudaStream_t st);
void launch_addsub(const KernelEnv& env, u64* out, const u64* a, const u64* b, int limbs, size_t ps, int mode, cudaStream_t st,
                   int polys = 2);
void launch_add_const(const KernelEnv& env, u64* out, const u64* a, const ScalarArg& K, int limbs, size_t ps, cudaStream_t st,
                      int polys = 2);
void launch_mul_scalar(const KernelEnv& env, u64* out, const u64* a, const ScalarArg& K, int limbs, size_t ps, cudaStream_t st,
                       int polys = 2, int t0 = 0);
void launch_mul_plain(const KernelEnv& env, u64* out, const u64* a, const u64* pt, int limbs, size_t ps, cudaStream_t st,
                      int polys = 2);
// out[c][t] (+)= sum_i x_i[c][t] * K_i[t] for up to 16 terms; KR holds K_i times R
struct LincombArg {
    const u64* x[16];
    u64 KR[16][RK_MAX_PRIMES];
};
void launch_lincomb(const KernelEnv& env, u64* out, const LincombArg& a, int terms, bool accumulate, int limbs, size_t ps,
                    cudaStream_t st, int polys = 2);
void launch_tensor(const KernelEnv& env, u64* d, const u64* x, const u64* y, int limbs, size_t ps, cudaStream_t st, int B = 1);
void launch_modup(const KernelEnv& env, const u64* x, const u64* x_eval, size_t eval_stride, u64* ext, size_t ext_stride,
                  int level, int beta, cudaStream_t st, int B = 1);
void launch_moddown_conv(const KernelEnv& env, const u64* u, u64* w, int level, cudaStream_t st, int polys = 2);
// a product's ModDown fused with its rescale (sources q_l and P, targets q_0 .. q_(l-1))
void launch_moddown_rs_conv(const KernelEnv& env, const u64* u, u64* w, int level, cudaStream_t st, int polys);
void launch_ks_add_pd(const KernelEnv& env, u64* u, const u64* d, int level, u64 pm, u64 pm_sh, cudaStream_t st, int B);
void launch_ks_combine_rs(const KernelEnv& env, u64* out, size_t ps, const u64* u, const u64* w, const u64* d, int level,
                          cudaStream_t st, int B);

// accumulate: add the products to the sums already in u (a hoisted sum of rotations)
void launch_ks_inner(const KernelEnv& env, const u64* ext, size_t ext_stride, KeyRef key, u64* u, int level, int beta,
                     u64 galois, cudaStream_t st, int B = 1, bool accumulate = false);
// Galois elements of a hoisted sum of up to three rotations
struct GaloisSet {
    int K;
    u64 g[3];
};
void launch_ks_combine_sum(const KernelEnv& env, u64* out, size_t ps, const u64* x, size_t bstride, const GaloisSet& gs,
                           bool add, const u64* u, const u64* w, int level, cudaStream_t st, int B);
void launch_ks_combine(const KernelEnv& env, u64* out, size_t ps, const u64* base0, u64 galois0, const u64* base1, size_t bstride,
                       const u64* u, const u64* w, int level, cudaStream_t st, int B = 1, const u64* addend = nullptr);
// fused key switching (ks_fused.cu)
void ks_fused_init_attributes();
void launch_modup_col(const KernelEnv& env, const u64* coef, u64* ext, size_t ext_stride, int level, int beta, int t0, int limbs,
                      cudaStream_t st, int B = 1, const u64* x_eval = nullptr, size_t eval_stride = 0);
// the row pass of a forward NTT whose column pass ran elsewhere (k_modup_col)
void launch_ntt_forward_rows(const KernelEnv& env, const LimbSet& s, cudaStream_t st);
void launch_ks_row(const KernelEnv& env, const u64* ext, size_t ext_stride, const u64* x_eval, size_t eval_stride, KeyRef key,
                   u64* u, int level, int beta, int t0, int limbs, u64 galois, cudaStream_t st, int B = 1);
void launch_moddown_col(const KernelEnv& env, const u64* u, u64* w, int level, cudaStream_t st, int polys = 2);
void launch_moddown_row(const KernelEnv& env, u64* out, size_t ps, const u64* base0, u64 galois0, const u64* base1, size_t bstride,
                        const u64* u, const u64* w, int level, cudaStream_t st, int B = 1);
void launch_rescale_lift(const KernelEnv& env, const u64* last, size_t ls, u64* v, int level, cudaStream_t st, int polys = 2);
void launch_rescale_combine(const KernelEnv& env, u64* ct, size_t ps, const u64* v, int level, cudaStream_t st, int polys = 2);
// out = (K in - v) q_l^-1 on limbs < level; K null for K = 1
void launch_rescale_combine(const KernelEnv& env, u64* out, const u64* in, size_t ps, const u64* v, int level, const ScalarArg* K,
                            cudaStream_t st, int polys);
void launch_reduce_signed(const KernelEnv& env, const int64_t* src, const LimbSet& s, cudaStream_t st);
void launch_uniform(const KernelEnv& env, const LimbSet& s, u64 seed, u64 stream_id, cudaStream_t st);
void launch_key_digit(const KernelEnv& env, u64* kb, u64* ka, const u64* a, const u64* e, const u64* s_R, const u64* sp,
                      const u64* gad_dev, int n_primes, cudaStream_t st);
void launch_key_digit_seeded(const KernelEnv& env, u64* kb, const u64* e, const u64* s_R, const u64* sp, const u64* gad_dev,
                             u64 seed, int j, int n_primes, cudaStream_t st);
void launch_to_mont(const KernelEnv& env, const LimbSet& s, cudaStream_t st);
void launch_automorph(const KernelEnv& env, u64* out, const u64* x, u64 g, int limbs, cudaStream_t st);
void launch_decrypt(const KernelEnv& env, u64* m, const u64* c0, const u64* c1, const u64* s_R, int limbs, cudaStream_t st);
void launch_encrypt(const KernelEnv& env, u64* ct, size_t ps, const u64* r, const u64* pk, size_t pk_ps, int limbs, cudaStream_t st);
void launch_pk(const KernelEnv& env, u64* pk, size_t ps, const u64* a, const u64* e, const u64* s_R, int limbs, cudaStream_t st);
void launch_square_secret(const KernelEnv& env, u64* out, const u64* s_R, int limbs, cudaStream_t st);
void launch_from_mont(const KernelEnv& env, u64* out, const u64* x, int limbs, cudaStream_t st);
