// Context creation: prime chain, canonical scales, NTT twiddles and the constant
// tables of the RNS basis conversions (Sec. 2.1 scheme substrate).
#include <atomic>
#include <cmath>
#include <cstring>

#include "kernels.cuh"

// ---------------------------------------------------------------------------
// Host number theory
// ---------------------------------------------------------------------------
u64 h_mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }

u64 h_powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = h_mulmod(r, a, q);
        a = h_mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

u64 h_invmod(u64 a, u64 q) { return h_powmod(a, q - 2, q); }

static bool h_is_prime(u64 n) {
    if (n < 2) return false;
    static const u64 small[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : small) {
        if (n == p) return true;
        if (n % p == 0) return false;
    }
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        s++;
    }
    for (u64 a : small) {
        u64 x = h_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int r = 1; r < s && witness; r++) {
            x = h_mulmod(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

int64_t round_half_away(double x) { return (int64_t)llround(x); }

static bool in_list(const std::vector<u64>& v, u64 x) {
    for (u64 y : v)
        if (y == x) return true;
    return false;
}

// largest prime < bound with p = 1 mod m, not in `used`
static u64 largest_prime_below(u64 bound, u64 m, const std::vector<u64>& used) {
    u64 k = (bound - 2) / m;
    for (;; k--) {
        u64 c = k * m + 1;
        if (!in_list(used, c) && h_is_prime(c)) return c;
    }
}

// prime p = 1 mod m nearest to c (ties to the smaller), not in `used`
static u64 nearest_prime(u64 c, u64 m, const std::vector<u64>& used) {
    u64 lo = ((c - 1) / m) * m + 1;
    u64 hi = lo + m;
    for (;;) {
        if (c - lo <= hi - c) {
            if (lo > 2 && !in_list(used, lo) && h_is_prime(lo)) return lo;
            lo -= m;
        } else {
            if (!in_list(used, hi) && h_is_prime(hi)) return hi;
            hi += m;
        }
    }
}

// primitive 2n-th root of unity mod q: c^((q-1)/2n) of the first c = 2, 3, ... of order 2n
static u64 root_2n(u64 q, u64 two_n) {
    for (u64 c = 2;; c++) {
        u64 w = h_powmod(c, (q - 1) / two_n, q);
        if (h_powmod(w, two_n / 2, q) == q - 1) return w;
    }
}

static u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

static u64 mont_qinv(u64 q) {  // q^-1 mod 2^64 by Newton iteration
    u64 x = q;                 // correct to 3 bits for odd q
    for (int i = 0; i < 6; i++) x *= 2 - q * x;
    return x;
}

static int bitrev(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

static std::atomic<uint64_t> g_device_allocs{0};
uint64_t rk_alloc_counted() { return g_device_allocs.load(); }
// Freed stream-ordered allocations stay reserved in the device's default pool (its
// release threshold is raised at context creation), and blocks of other sizes do not
// serve a request; so when an allocation fails, the unused reserve is returned to the
// device and the allocation is tried once more.
static cudaError_t trim_and_retry(cudaError_t e, cudaStream_t st) {
    if (e != cudaErrorMemoryAllocation) return e;
    cudaGetLastError();   // clear the failed allocation's error
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return e;
    if (st) {   // not while a graph is being captured on the stream
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return e;
        cudaStreamSynchronize(st);
    }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess || cudaMemPoolTrimTo(pool, 0) != cudaSuccess) return e;
    return cudaSuccess;
}
cudaError_t rk_malloc(void** p, size_t bytes) {
    g_device_allocs++;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation && trim_and_retry(e, nullptr) == cudaSuccess) e = cudaMalloc(p, bytes);
    return e;
}
cudaError_t rk_malloc_async(void** p, size_t bytes, cudaStream_t st) {
    g_device_allocs++;
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e == cudaErrorMemoryAllocation && trim_and_retry(e, st) == cudaSuccess) e = cudaMallocAsync(p, bytes, st);
    return e;
}

u64* rk_ctx::scratch(size_t words) {
    if (words > scratch_words) {
        RK_CUDA(cudaStreamSynchronize(stream));
        if (d_scratch) RK_CUDA(cudaFree(d_scratch));
        generation++;
        d_scratch = nullptr;
        RK_CUDA(rk_malloc((void**)&d_scratch, words * 8));
        scratch_words = words;
    }
    return d_scratch;
}

static void validate(const rk_params* p) {
    RK_REQUIRE(p, RK_EINVAL, "params is NULL");
    RK_REQUIRE(p->log_n >= 10 && p->log_n <= 17, RK_EINVAL, "log_n must be in [10, 17]");
    RK_REQUIRE(p->n_limbs >= 1 && p->n_special >= 1 && p->n_special <= RK_MAX_SPECIAL, RK_EINVAL, "bad limb counts");
    RK_REQUIRE(p->n_limbs + p->n_special <= RK_MAX_PRIMES, RK_EINVAL, "too many primes");
    RK_REQUIRE(p->digit_size >= 1 && p->digit_size <= RK_MAX_DIGIT, RK_EINVAL, "digit_size must be in [1, 8]");
    RK_REQUIRE(p->cmp_cheb == 0 || (p->cmp_cheb >= 4 && p->cmp_cheb <= 16384 && (p->cmp_cheb & (p->cmp_cheb - 1)) == 0),
               RK_EINVAL, "cmp_cheb must be 0 or a power of two in [4, 16384]");
    RK_REQUIRE((p->n_limbs + p->digit_size - 1) / p->digit_size <= 16, RK_EINVAL, "at most 16 key-switching digits");
    RK_REQUIRE(p->log_scale >= 20 && p->log_scale <= 58, RK_EINVAL, "log_scale must be in [20, 58]");
    RK_REQUIRE(p->log_q0 >= 20 && p->log_q0 <= 61, RK_EINVAL, "log_q0 must be in [20, 61]");
    RK_REQUIRE(p->log_special >= 20 && p->log_special <= 61, RK_EINVAL, "log_special must be in [20, 61]");
    RK_REQUIRE(p->prime_form <= 1, RK_EINVAL, "prime_form must be 0 or 1");
    RK_REQUIRE(p->prime_form == 0 || (p->log_scale >= 34 && p->log_q0 >= 34 && p->log_special >= 34), RK_EINVAL,
               "prime_form 1 (primes k 2^32 + 1) needs log_scale, log_q0 and log_special of at least 34");
}

// The prime chain and canonical scales of a parameter set (host only, no device):
// q_0..q_L then the special primes, and Delta_0..Delta_L.
void params_chain(const rk_params* p, std::vector<u64>& primes, std::vector<double>& scales) {
    validate(p);
    const int n = 1 << p->log_n, L = (int)p->n_limbs - 1, alpha = (int)p->n_special;
    const u64 m = 2ull * (u64)n;
    // candidate step: primes = 1 mod 2n, or (prime_form 1) = 1 mod 2^32, which 2n divides
    const u64 step = p->prime_form ? (1ull << 32) : m;
    std::vector<u64> used;
    std::vector<u64> q(L + 1);
    q[0] = largest_prime_below(1ull << p->log_q0, step, used);
    used.push_back(q[0]);
    std::vector<double> sc(L + 1);
    const double two_ls = std::ldexp(1.0, (int)p->log_scale);
    sc[L] = two_ls;
    for (int l = L; l >= 1; l--) {
        volatile double t = sc[l] * sc[l];
        double target = t / two_ls;
        u64 ql = nearest_prime((u64)std::floor(target), step, used);
        used.push_back(ql);
        q[l] = ql;
        volatile double sq = sc[l] * sc[l];
        sc[l - 1] = sq / (double)ql;
    }
    u64 bound = 1ull << p->log_special;
    primes = q;
    for (int k = 0; k < alpha; k++) {
        u64 pk = largest_prime_below(bound, step, used);
        used.push_back(pk);
        primes.push_back(pk);
        bound = pk;
    }
    scales = sc;
    for (u64 x : primes) RK_REQUIRE(x < (1ull << 61), RK_EINVAL, "prime above 2^61");
}

void ctx_build(rk_ctx* c, const rk_params* p, int device, void* stream) {
    validate(p);
    c->prm = *p;
    c->device = device;
    RK_CUDA(cudaSetDevice(device));
    if (stream) {
        c->stream = (cudaStream_t)stream;
        c->own_stream = false;
    } else {
        RK_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    {   // keep freed stream-ordered allocations in the pool
        cudaMemPool_t pool;
        RK_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
        uint64_t thr = UINT64_MAX;
        RK_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    }
    c->log_n = (int)p->log_n;
    c->n = 1 << c->log_n;
    c->L = (int)p->n_limbs - 1;
    c->alpha = (int)p->n_special;
    c->dsize = (int)p->digit_size;
    c->n_primes = c->L + 1 + c->alpha;
    const u64 m = 2ull * (u64)c->n;

    // ---- prime chain and canonical scales ----
    params_chain(p, c->primes, c->scales);
    const std::vector<u64> q(c->primes.begin(), c->primes.begin() + c->L + 1);
    const std::vector<u64> sp(c->primes.begin() + c->L + 1, c->primes.end());

    // ---- per-prime constants ----
    const int NP = c->n_primes, n = c->n;
    c->h_pc.resize(NP);
    for (int i = 0; i < NP; i++) {
        u64 qi = c->primes[i];
        PrimeConst& P = c->h_pc[i];
        P.q = qi;
        P.qinv = mont_qinv(qi);
        P.r_mod = (u64)(((u128)1 << 64) % qi);
        P.r2 = h_mulmod(P.r_mod, P.r_mod, qi);
        P.r_shoup = shoup_of(P.r_mod, qi);
        P.ninv = h_invmod((u64)n % qi, qi);
        P.ninv_shoup = shoup_of(P.ninv, qi);
        P.one_shoup = shoup_of(1, qi);
    }
    RK_CUDA(rk_malloc((void**)&c->d_pc, NP * sizeof(PrimeConst)));
    RK_CUDA(cudaMemcpy(c->d_pc, c->h_pc.data(), NP * sizeof(PrimeConst), cudaMemcpyHostToDevice));

    // ---- twiddles: (psi^brev(i), Shoup companion) and (psi^-brev(i), companion) pairs ----
    std::vector<u64> tw((size_t)4 * NP * n);
    for (int i = 0; i < NP; i++) {
        u64 qi = c->primes[i];
        u64 psi = root_2n(qi, m), ipsi = h_invmod(psi, qi);
        std::vector<u64> pw(n), ipw(n);
        pw[0] = ipw[0] = 1;
        for (int k = 1; k < n; k++) {
            pw[k] = h_mulmod(pw[k - 1], psi, qi);
            ipw[k] = h_mulmod(ipw[k - 1], ipsi, qi);
        }
        u64* F = tw.data() + (size_t)i * 2 * n;              // forward pairs
        u64* I = tw.data() + ((size_t)NP + i) * 2 * n;       // inverse pairs
        for (int k = 0; k < n; k++) {
            int r = bitrev(k, c->log_n);
            F[2 * k] = pw[r];
            F[2 * k + 1] = shoup_of(pw[r], qi);
            I[2 * k] = ipw[r];
            I[2 * k + 1] = shoup_of(ipw[r], qi);
        }
    }
    RK_CUDA(rk_malloc((void**)&c->d_tw, tw.size() * 8));
    RK_CUDA(cudaMemcpy(c->d_tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice));

    // ---- basis conversion constants ----
    const int L = c->L, A = c->alpha, DS = c->dsize, T = L + 1 + A;
    const int beta_max = c->beta(L);
    const size_t mu_stride = (size_t)2 * DS + (size_t)DS * T;
    std::vector<u64> conv;
    // ModUp blocks
    const size_t mu_off = 0;
    conv.resize(mu_off + (size_t)(L + 1) * beta_max * mu_stride, 0);
    for (int l = 0; l <= L; l++) {
        for (int j = 0; j < c->beta(l); j++) {
            u64* blk = conv.data() + mu_off + ((size_t)l * beta_max + j) * mu_stride;
            int lo = j * DS, hi = std::min(lo + DS, l + 1);
            for (int i = lo; i < hi; i++) {
                u64 qi = q[i];
                u64 dh = 1;
                for (int i2 = lo; i2 < hi; i2++)
                    if (i2 != i) dh = h_mulmod(dh, q[i2] % qi, qi);
                u64 inv = h_invmod(dh, qi);
                blk[i - lo] = inv;
                blk[DS + (i - lo)] = shoup_of(inv, qi);
                for (int t = 0; t < l + 1 + A; t++) {
                    int pid = t <= l ? t : L + 1 + (t - l - 1);
                    u64 pt = c->primes[pid];
                    u64 v = 1 % pt;
                    for (int i2 = lo; i2 < hi; i2++)
                        if (i2 != i) v = h_mulmod(v, q[i2] % pt, pt);
                    blk[2 * DS + (size_t)(i - lo) * T + t] = h_mulmod(v, c->h_pc[pid].r_mod, pt);
                }
            }
        }
    }
    // ModDown block
    const size_t md_off = conv.size();
    conv.resize(md_off + 2 * A + (size_t)A * (L + 1) + (L + 1), 0);
    for (int i = 0; i <= L; i++) {   // P mod q_i, subtracted once per negative centred term
        u64 pm = 1 % q[i];
        for (int k = 0; k < A; k++) pm = h_mulmod(pm, sp[k] % q[i], q[i]);
        conv[md_off + 2 * A + (size_t)A * (L + 1) + i] = pm;
    }
    for (int k = 0; k < A; k++) {
        u64 pk = sp[k];
        u64 ph = 1;
        for (int k2 = 0; k2 < A; k2++)
            if (k2 != k) ph = h_mulmod(ph, sp[k2] % pk, pk);
        u64 inv = h_invmod(ph, pk);
        conv[md_off + k] = inv;
        conv[md_off + A + k] = shoup_of(inv, pk);
        for (int i = 0; i <= L; i++) {
            u64 v = 1 % q[i];
            for (int k2 = 0; k2 < A; k2++)
                if (k2 != k) v = h_mulmod(v, sp[k2] % q[i], q[i]);
            conv[md_off + 2 * A + (size_t)k * (L + 1) + i] = h_mulmod(v, c->h_pc[i].r_mod, q[i]);
        }
    }
    // P^-1 mod q_i
    const size_t pi_off = conv.size();
    conv.resize(pi_off + 2 * (size_t)(L + 1), 0);
    c->h_pinv.resize(L + 1);
    for (int i = 0; i <= L; i++) {
        u64 pm = 1;
        for (int k = 0; k < A; k++) pm = h_mulmod(pm, sp[k] % q[i], q[i]);
        u64 inv = h_invmod(pm, q[i]);
        conv[pi_off + 2 * i] = inv;
        conv[pi_off + 2 * i + 1] = shoup_of(inv, q[i]);
        c->h_pinv[i] = inv;
    }
    // rescale blocks
    const size_t rs_off = conv.size();
    conv.resize(rs_off + (size_t)(L + 1) * 3 * (L + 1), 0);
    for (int l = 1; l <= L; l++) {
        u64* blk = conv.data() + rs_off + (size_t)l * 3 * (L + 1);
        for (int i = 0; i < l; i++) {
            u64 inv = h_invmod(q[l] % q[i], q[i]);
            blk[i] = inv;
            blk[(L + 1) + i] = shoup_of(inv, q[i]);
            blk[2 * (L + 1) + i] = q[l] % q[i];
        }
    }
    // fused ModDown + rescale blocks
    const size_t A1 = (size_t)A + 1, rs_stride = 2 * A1 + A1 * (L + 1) + 3 * (size_t)(L + 1) + A1;
    const size_t mr_off = conv.size();
    conv.resize(mr_off + (size_t)(L + 1) * rs_stride, 0);
    for (int l = 1; l <= L; l++) {
        u64* blk = conv.data() + mr_off + (size_t)l * rs_stride;
        std::vector<u64> src(1, q[l]);
        for (int k = 0; k < A; k++) src.push_back(sp[k]);
        for (size_t k = 0; k < A1; k++) {
            const u64 sk = src[k];
            u64 rest = 1 % sk;   // S / s_k mod s_k
            for (size_t k2 = 0; k2 < A1; k2++)
                if (k2 != k) rest = h_mulmod(rest, src[k2] % sk, sk);
            const u64 inv = h_invmod(rest, sk);
            blk[k] = inv;
            blk[A1 + k] = shoup_of(inv, sk);
            for (int i = 0; i < l; i++) {
                u64 v = 1 % q[i];
                for (size_t k2 = 0; k2 < A1; k2++)
                    if (k2 != k) v = h_mulmod(v, src[k2] % q[i], q[i]);
                blk[2 * A1 + k * (L + 1) + i] = h_mulmod(v, c->h_pc[i].r_mod, q[i]);
            }
        }
        u64* smod = blk + 2 * A1 + A1 * (L + 1);
        for (int i = 0; i < l; i++) {
            u64 v = 1 % q[i];
            for (size_t k = 0; k < A1; k++) v = h_mulmod(v, src[k] % q[i], q[i]);
            smod[i] = v;
            const u64 inv = h_invmod(v, q[i]);
            smod[(L + 1) + i] = inv;
            smod[2 * (L + 1) + i] = shoup_of(inv, q[i]);
        }
        double* rcp = reinterpret_cast<double*>(smod + 3 * (L + 1));   // 1 / s_k, correctly rounded
        for (size_t k = 0; k < A1; k++) rcp[k] = 1.0 / (double)src[k];
    }
    RK_CUDA(rk_malloc((void**)&c->d_conv, conv.size() * 8));
    RK_CUDA(cudaMemcpy(c->d_conv, conv.data(), conv.size() * 8, cudaMemcpyHostToDevice));

    KernelEnv& e = c->env;
    e.logn = c->log_n;
    e.n = n;
    e.L = L;
    e.alpha = A;
    e.pc = c->d_pc;
    e.sp = true;
    for (u64 x : c->primes) e.sp = e.sp && is_k32_prime(x);
    e.tw.psi = c->d_tw;
    e.tw.ipsi = c->d_tw + (size_t)2 * NP * n;
    e.conv.modup = c->d_conv + mu_off;
    e.conv.modup_stride = mu_stride;
    e.conv.beta_max = beta_max;
    e.conv.dsize = DS;
    e.conv.moddown = c->d_conv + md_off;
    e.conv.pinv = c->d_conv + pi_off;
    e.conv.rescale = c->d_conv + rs_off;
    e.conv.mdrs = c->d_conv + mr_off;
    e.conv.mdrs_stride = rs_stride;
    e.prof = &c->prof;
    e.tune = &c->tune;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) == cudaSuccess && sms > 0) e.sms = sms;
    ntt_init_attributes();
    ks_fused_init_attributes();
}

void server_stop(rk_ctx* c);

// An execution lane of `parent` for the serving loop: the parent's parameters, device
// tables, keys, encodings and coefficients (shared, read only, never freed through the
// lane), with a stream, a scratch area, plaintext caches and a profiler of its own, so
// that circuits on different lanes run concurrently on the device.
rk_ctx* ctx_lane_create(rk_ctx* parent) {
    rk_ctx* c = new rk_ctx();
    c->lane_of = parent;
    c->prm = parent->prm;
    c->device = parent->device;
    c->log_n = parent->log_n;
    c->n = parent->n;
    c->L = parent->L;
    c->alpha = parent->alpha;
    c->dsize = parent->dsize;
    c->n_primes = parent->n_primes;
    c->primes = parent->primes;
    c->scales = parent->scales;
    c->ninv = parent->ninv;
    c->d_tw = parent->d_tw;
    c->d_conv = parent->d_conv;
    c->d_pc = parent->d_pc;
    c->h_pc = parent->h_pc;
    c->h_pinv = parent->h_pinv;
    c->d_sk = parent->d_sk;
    c->h_sk = parent->h_sk;
    c->d_pk = parent->d_pk;
    c->rlk = parent->rlk;
    c->gal = parent->gal;
    c->seed = parent->seed;
    c->tune = parent->tune;
    c->ks_fused = parent->ks_fused;
    c->modup_col = parent->modup_col;
    c->stack_blocks = parent->stack_blocks;
    c->trim_levels = parent->trim_levels;
    c->pair_packing = parent->pair_packing;
    c->ks_group_bytes = parent->ks_group_bytes;
    c->ind_stack_bytes = parent->ind_stack_bytes;
    c->stack_budget_bytes = parent->stack_budget_bytes;
    c->cmp_coeffs = parent->cmp_coeffs;
    c->encodings = parent->encodings;
    c->indicator = parent->indicator;
    c->env = parent->env;
    c->env.prof = &c->prof;
    c->env.tune = &c->tune;
    try {
        RK_CUDA(cudaSetDevice(c->device));
        RK_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    } catch (...) {
        delete c;
        throw;
    }
    return c;
}

// Frees what the lane owns (stream, scratch, cached plaintexts, events) and the lane.
void ctx_lane_release(rk_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& kv : c->plain_cache) cudaFree(kv.second);
    for (auto& kv : c->plain_add_cache) cudaFree(kv.second);
    if (c->d_scratch) cudaFree(c->d_scratch);
    for (cudaEvent_t ev : c->prof.ev) cudaEventDestroy(ev);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

void ctx_release(rk_ctx* c) {
    if (!c) return;
    server_stop(c);
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& kv : c->plain_cache) cudaFree(kv.second);
    for (auto& kv : c->plain_add_cache) cudaFree(kv.second);
    for (auto& kv : c->gal) cudaFree(kv.second.data);
    if (c->rlk.data) cudaFree(c->rlk.data);
    if (c->d_sk) cudaFree(c->d_sk);
    if (c->d_pk) cudaFree(c->d_pk);
    if (c->d_scratch) cudaFree(c->d_scratch);
    if (c->d_conv) cudaFree(c->d_conv);
    if (c->d_tw) cudaFree(c->d_tw);
    if (c->d_pc) cudaFree(c->d_pc);
    for (cudaEvent_t ev : c->prof.ev) cudaEventDestroy(ev);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}
