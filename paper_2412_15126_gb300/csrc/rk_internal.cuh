// Internal declarations of the CUDA RNS-CKKS library behind include/rankfhe.h.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/rankfhe.h"
#include "modarith.cuh"

// ---------------------------------------------------------------------------
// Errors: internal code throws rk_error; the C-ABI converts to rk_status.
// ---------------------------------------------------------------------------
struct rk_error : std::runtime_error {
    rk_status code;
    rk_error(rk_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};
#define RK_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t _e = (call);                                                            \
        if (_e != cudaSuccess)                                                              \
            throw rk_error(RK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e));   \
    } while (0)
#define RK_REQUIRE(cond, code, msg)                  \
    do {                                             \
        if (!(cond)) throw rk_error((code), (msg));  \
    } while (0)

// Every device allocation of the library goes through these two, which count the
// calls (rk_device_alloc_count reports the total).
uint64_t rk_alloc_counted();
cudaError_t rk_malloc(void** p, size_t bytes);
cudaError_t rk_malloc_async(void** p, size_t bytes, cudaStream_t st);

// ---------------------------------------------------------------------------
// Device-side description of a set of residue polynomials.
// Limb t of poly p lives at base + p * poly_stride + t * n.
// Limb t uses prime id  t < split ? t + off_lo : off_hi + (t - split).
// ---------------------------------------------------------------------------
struct LimbSet {
    u64* base;
    size_t poly_stride;
    int n_polys;
    int n_limbs;
    int split;
    int off_lo;
    int off_hi;
    // optional: skip limbs t < split with t / skip_ds == poly % skip_beta (the lifted
    // digits of a ModUp already hold their own limbs in the evaluation domain)
    int skip_ds = 0;
    int skip_beta = 1;
    // optional: an inverse NTT's first pass reads polynomial z from src + z * src_stride
    // (same limb layout) instead of transforming base in place
    const u64* src = nullptr;
    size_t src_stride = 0;
    // optional (rescale): a forward NTT's first pass reads, for polynomial z, the one
    // coefficient-domain limb lift + z * lift_stride, residues modulo lift_q, and takes
    // its centred representative modulo each limb's prime; lift_mod[t] = lift_q mod
    // prime(t)
    const u64* lift = nullptr;
    size_t lift_stride = 0;
    const u64* lift_mod = nullptr;
    u64 lift_q = 0;
    // NTT launches over a group of the limbs: grid z covers limbs limb0 .. limb0 +
    // n_limbs - 1 of the set (limb indices stay those of the whole set)
    int limb0 = 0;
};

__host__ __device__ __forceinline__ int limb_prime(const LimbSet& s, int t) {
    return t < s.split ? t + s.off_lo : s.off_hi + (t - s.split);
}

// Per-level constants of the basis conversions (device memory, see context.cu).
struct ConvTables {
    // ModUp, for level l and digit j: block at modup + (l * beta_max + j) * modup_stride:
    //   [0, DS)           (D/q_i)^-1 mod q_i          (source i of the digit)
    //   [DS, 2DS)         Shoup companions
    //   [2DS, 2DS + DS*T) (D/q_i) mod prime(t) times R, t = 0 .. l+alpha, row-major [i][t]
    //   T = L + 1 + alpha is the row length (only the first l+1+alpha columns are used)
    const u64* modup;
    size_t modup_stride;
    int beta_max;
    int dsize;
    // ModDown (level independent): [0, A) (P/p_k)^-1 mod p_k, [A, 2A) Shoup,
    //   [2A, 2A + A*(L+1)) (P/p_k) mod q_i times R, row-major [k][i],
    //   then (L+1) words P mod q_i
    const u64* moddown;
    // P^-1 mod q_i and Shoup companion: [2 * (L+1)]
    const u64* pinv;
    // Rescale for level l: block at rescale + l * 3 * (L+1):
    //   [0, L+1) q_l^-1 mod q_i; [L+1, 2(L+1)) Shoup; [2(L+1), 3(L+1)) q_l mod q_i
    const u64* rescale;
    // ModDown fused with the rescale of a product at level l (S = q_l P, sources
    // s_0 = q_l, s_(k+1) = p_k): block at mdrs + l * mdrs_stride:
    //   [0, A+1) (S/s_k)^-1 mod s_k, [A+1, 2(A+1)) Shoup,
    //   [2(A+1), 2(A+1) + (A+1)(L+1)) (S/s_k) mod q_i times R, row-major [k][i],
    //   then (L+1) words S mod q_i, then (L+1) words S^-1 mod q_i and (L+1) Shoup,
    //   then A+1 doubles 1/s_k (the rounded conversion's reciprocals)
    const u64* mdrs;
    size_t mdrs_stride;
};

struct DevTables {
    const u64* psi;       // [n_primes][n][2]  (psi^brev(i), its Shoup companion)
    const u64* ipsi;      // [n_primes][n][2]  (psi^-brev(i), its Shoup companion)
};

// Constants of a scalar multiplication (one residue per limb, with Shoup companions).
struct ScalarArg {
    u64 w[RK_MAX_PRIMES];
    u64 wsh[RK_MAX_PRIMES];
};

#define RK_MAX_DIGIT 8
#define RK_MAX_SPECIAL 8

// Kernel kinds the profiler can time (rk_profile_start names).
enum KernelKind {
    KK_NTT_FWD = 0, KK_NTT_INV, KK_MODUP, KK_KS_INNER, KK_MODDOWN, KK_KS_COMBINE, KK_TENSOR, KK_RESCALE,
    KK_POINTWISE, KK_CLIENT, KK_COUNT
};
extern const char* const kKernelKindNames[KK_COUNT];

// Launch counter and CUDA-event timing of one kernel kind on the context stream.
struct Profiler {
    uint64_t launches = 0;        // every kernel this library launched
    uint32_t mask = 0;            // kinds being timed (bit k for kind k), 0 = none
    bool paused = false;          // timing suspended (rk_profile_pause)
    std::vector<cudaEvent_t> ev;  // start/stop pairs
    std::vector<int> ev_kind;     // kind of each pair
    size_t used = 0;
    // per kind, since the last rk_profile_start: algorithmic bytes, modular products,
    // timed launches; milliseconds once rk_profile_stop has read the events
    double bytes[KK_COUNT] = {}, ops[KK_COUNT] = {}, ms[KK_COUNT] = {};
    uint64_t timed[KK_COUNT] = {};
};

// Everything a kernel launcher needs: sizes and device tables.
// Mask kinds whose n_real argument is part of the plaintext (padding length or the
// denominator of a scaled mask); the others ignore it.
inline uint32_t mask_nreal(uint32_t kind, uint32_t n_real) {
    return (kind == RK_MASK_VALID || kind == RK_MASK_ROW0S || kind == RK_MASK_COL0S || kind == RK_MASK_ROWIDX) ? n_real : 0;
}

// Launch shapes chosen by rk_autotune (0 keeps the built-in rule).  NTT block widths
// (transforms per block) indexed [inverse][column pass][small: fewer than 16 limbs].
struct TuneTable {
    int ntt_units[2][2][2] = {};
    // a forward or inverse NTT of more bytes than this runs as limb groups of at most
    // this size, both passes of one group before the next (the intermediate between
    // the passes then stays in L2); 0: one launch pair for the whole set
    size_t ntt_group_bytes = 0;
};

struct KernelEnv {
    int logn, n, L, alpha;
    int sms = 152;          // multiprocessors of the device (grid sizing)
    bool sp = false;        // every prime is k 2^32 + 1 (kernels take the cheaper products by q)
    const TuneTable* tune = nullptr;
    const PrimeConst* pc;   // device array [n_primes]
    DevTables tw;
    ConvTables conv;
    Profiler* prof;
};

// ---------------------------------------------------------------------------
// Host context
// ---------------------------------------------------------------------------
struct DevBuf {
    u64* p = nullptr;
    size_t words = 0;
};

// A switching key on the device, evaluation domain, Montgomery form, T = L+1+alpha
// primes: data = [beta_L][2][T][n] (b_j then a_j), or, seeded, [beta_L][1][T][n] (b_j
// only) with a_j regenerated from `seed` (seeded_key_word).
struct KeyRef {
    const u64* data;
    u64 seed;
    int seeded;
};

// Seeded key halves: SplitMix64 (Steele, Lea and Flood 2014) from its published
// definition.  Element c of the stream from seed s is sm64_mix(s + (c + 1) GAMMA);
// word (digit j, prime index p, evaluation index k) of a key's a part is element
// (j T + p) n + k, and its value in [0, q_p), the high word of x q_p, is the
// Montgomery form a 2^64 mod q_p.
constexpr u64 kSm64Gamma = 0x9E3779B97F4A7C15ull;
__host__ __device__ __forceinline__ u64 sm64_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// state of word (j, p, k): seed + ((j T + p) n + k + 1) GAMMA
__host__ __device__ __forceinline__ u64 seeded_key_state(u64 seed, int j, int T, int p, int n, int k) {
    return seed + ((((u64)j * (u64)T + (u64)p) * (u64)n + (u64)k) + 1) * kSm64Gamma;
}
__device__ __forceinline__ u64 seeded_key_word(u64 state, u64 q) { return umulhi64(sm64_mix(state), q); }
template <bool SP>
__device__ __forceinline__ u64 seeded_key_word_t(u64 state, u64 q) {
    return SP ? mulhi_q_k32(sm64_mix(state), q) : umulhi64(sm64_mix(state), q);
}

struct SwitchKeyDev {
    u64* data = nullptr;  // [beta_L][2][L+1+alpha][n] (seeded: [beta_L][1][..][n], b only),
                          // evaluation domain, Montgomery form
    u64 seed = 0;         // seeded: the a parts are regenerated from this seed
    bool seeded = false;
    KeyRef ref() const { return KeyRef{data, seed, seeded ? 1 : 0}; }
};

struct rk_server;

struct rk_ctx {
    rk_params prm{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int log_n = 0, n = 0, L = 0, alpha = 0, dsize = 0, n_primes = 0;
    std::vector<u64> primes;      // q_0..q_L, p_0..p_{alpha-1}
    std::vector<double> scales;   // Delta_0..Delta_L
    std::vector<u64> ninv;        // n^-1 mod prime
    // device tables
    u64* d_tw = nullptr;          // 4 * n_primes * n
    u64* d_conv = nullptr;
    PrimeConst* d_pc = nullptr;
    std::vector<PrimeConst> h_pc;
    KernelEnv env{};
    Profiler prof;
    std::vector<u64> h_pinv;      // host copies used by the encoder/decoder
    // keys (device)
    u64* d_sk = nullptr;          // secret in eval domain over all primes, Montgomery form
    std::vector<int64_t> h_sk;    // secret coefficients (ternary)
    u64* d_pk = nullptr;          // [2][L+1][n] eval, Montgomery form
    SwitchKeyDev rlk;
    std::map<u64, SwitchKeyDev> gal;
    uint64_t enc_counter = 0;     // encryption randomness counter
    uint64_t seed = 0;
    // scratch (grows on demand; stream ordered)
    u64* d_scratch = nullptr;
    size_t scratch_words = 0;
    int batch_cap = 1;            // largest stack B the scratch layout is sized for
    rk_server* server = nullptr;  // serving loop, when one runs (it owns the stream meanwhile)
    rk_ctx* lane_of = nullptr;    // a serving lane: the context whose tables and keys it shares
    int server_lanes = 2;         // lanes (concurrent batches) of the next serving loop
    // Bumped whenever a buffer that captured CUDA graphs point into is replaced (scratch
    // growth, switching keys, cached plaintexts, indicator coefficients).
    uint64_t generation = 0;
    TuneTable tune;
    bool ks_fused = false;        // key switching with conversions fused into the NTT passes
    bool modup_col = false;       // staged key switching with the ModUp conversion fused into
                                  // the forward column pass (k_modup_col)
    bool stack_blocks = true;     // blocked rank: blocks and block pairs as stacks (else one by one)
    bool trim_levels = false;     // rank: bring the input down to the level the circuit needs first
    bool pair_packing = true;     // blocked circuits: pack block-pair work into free tiles when keys allow
    double ks_group_bytes = 48.0 * (1 << 20);   // lifted digits kept in L2 between the fused kernels
    size_t ind_stack_bytes = (size_t)4 << 30;   // working set of one stacked indicator evaluation
    size_t stack_budget_bytes = (size_t)16 << 30;   // working set of one stacked step of the blocked circuits
    u64* noalloc_scratch = nullptr;             // device address of the allocation-free rescale's array
    std::vector<double> cmp_coeffs;             // Chebyshev comparator coefficients (computed or imported)
    // plaintext caches: key = (kind, N, Q, n_real, level)
    std::map<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t, int>, u64*> plain_cache;
    std::map<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t>, std::vector<double>> encodings;
    // plaintexts for addition (scale Delta_l, normal form), same key
    std::map<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t, int>, u64*> plain_add_cache;
    // Chebyshev coefficients of the indicator window per padded length N
    std::map<uint32_t, std::vector<double>> indicator;
    // op counters
    uint64_t n_ks = 0, n_rot = 0, n_mul = 0, n_rescale = 0;
    size_t ct_words() const { return (size_t)2 * (L + 1) * n; }
    size_t poly_stride() const { return (size_t)(L + 1) * n; }
    int qp_limbs(int level) const { return level + 1 + alpha; }
    int beta(int level) const { return (level + 1 + dsize - 1) / dsize; }
    u64* scratch(size_t words);
};

struct rk_ct {
    rk_ctx* ctx = nullptr;
    u64* data = nullptr;   // [B][2][L+1][n] (only limbs 0..level are meaningful), evaluation domain
    int level = 0;
    int B = 1;             // ciphertexts stacked in this handle (one launch per operation for all)
    bool view = false;     // borrows `data` from another handle (never freed through this one)
    uint32_t N = 0;        // padded vector length (power of two)
    uint32_t n_real = 0;   // unpadded length
    uint32_t Q = 1;        // queries packed at stride N^2
    uint32_t layout = 0;   // RK_LAYOUT_ROW / RK_LAYOUT_COL
};

// ---------------------------------------------------------------------------
// Evaluator (evaluator.cu)
// ---------------------------------------------------------------------------
rk_ct* ct_alloc(rk_ctx* c, int level, int B = 1);
void ct_free(rk_ct* ct);
rk_ct* ct_clone_meta(const rk_ct* src, int level);
void ensure_batch(rk_ctx* c, int B);   // size the scratch for stacks of B ciphertexts
rk_ct* ct_stack(rk_ctx* c, const rk_ct* const* in, int count);        // B = count, copies
void ct_unstack(rk_ctx* c, const rk_ct* in, rk_ct** outs);            // B outputs of B = 1
void key_export(rk_ctx* c, const SwitchKeyDev& key, u64* host_out);
size_t key_words(const rk_ctx* c, const SwitchKeyDev& key);
rk_ct* ct_alloc_like(const rk_ct* like, int level, int B);   // vector metadata of `like`, B members
rk_ct* ct_view(const rk_ct* stack, int b);                            // member b, no copy
rk_ct* ct_view_range(const rk_ct* stack, int first, int count);      // members [first, first+count), no copy

void ev_add(rk_ctx* c, const rk_ct* a, const rk_ct* b, rk_ct* out);
void ev_sub(rk_ctx* c, const rk_ct* a, const rk_ct* b, rk_ct* out);
void ev_neg(rk_ctx* c, const rk_ct* a, rk_ct* out);
void ev_add_const(rk_ctx* c, const rk_ct* a, double v, rk_ct* out);
void ev_rescale_inplace(rk_ctx* c, rk_ct* a);
void ev_mul_scalar(rk_ctx* c, const rk_ct* a, double v, rk_ct* out);        // out at level-1
void ev_mul(rk_ctx* c, const rk_ct* a, const rk_ct* b, rk_ct* out);         // out at level-1
void ev_mul_pairs(rk_ctx* c, const rk_ct* const* a, const rk_ct* const* b, int n, rk_ct* out);   // stack of a[i] b[i]
void ev_mul_plain(rk_ctx* c, const rk_ct* a, uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real, rk_ct* out);
void ev_rotate_many(rk_ctx* c, const rk_ct* a, const int* r, int k, rk_ct** outs);  // left rotations
void ev_rotate_add(rk_ctx* c, const rk_ct* a, int r, rk_ct* out);               // a + (a <<< r)
void ev_rotate_multi(rk_ctx* c, const rk_ct* a, const int* r, bool add, rk_ct* out);  // member b by r[b]
// outs[s]_b = [a_b +] sum_k a_b <<< r[(s B + b) 3 + k], k < K[s] <= 3: one ModUp, one ModDown
void ev_rotate_sums(rk_ctx* c, const rk_ct* a, int nsets, const int* K, const int* r, bool add, rk_ct** outs);
void ev_add_plain(rk_ctx* c, const rk_ct* a, uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real, rk_ct* out);
void ev_lincomb(rk_ctx* c, const std::vector<const rk_ct*>& xs, const std::vector<double>& cs, rk_ct* out,
                bool rescale = true);   // sum c_i x_i, then a rescale unless told not to  // out at level-1
void ev_level_down(rk_ctx* c, const rk_ct* a, int target, rk_ct* out);
void ev_copy(rk_ctx* c, const rk_ct* a, rk_ct* out);

// keys / client ops
void keys_generate(rk_ctx* c, uint64_t seed, const std::vector<int>& rotations);
void keys_add_rotations(rk_ctx* c, const std::vector<int>& rotations);
void key_import(rk_ctx* c, uint32_t kind, uint64_t galois, const uint64_t* coeffs, size_t words, bool seeded = false,
                uint64_t seed = 0);
void secret_import(rk_ctx* c, const int64_t* s, size_t n);
u64 galois_left(const rk_ctx* c, int r);
rk_ct* encrypt_values(rk_ctx* c, const double* v, uint32_t count, uint32_t N, uint32_t Q, uint32_t n_real);
void decrypt_slots(rk_ctx* c, const rk_ct* ct, std::vector<double>& slots);
rk_ct* ct_import(rk_ctx* c, const uint64_t* coeffs, int level);
void ct_export(rk_ctx* c, const rk_ct* ct, uint64_t* coeffs);

// encoder (encoder.cpp)
void encode_unscaled(int log_n, const double* z, size_t count, std::vector<double>& u);
void decode_coeffs(int log_n, const std::vector<double>& m, std::vector<double>& slots);

// masks (circuits.cpp)
void mask_slot_values(uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real, size_t slots, std::vector<double>& v);
// the unscaled encoding of a mask the evaluator uses (its own FFT unless imported; evaluator.cu)
const std::vector<double>& encoding_of(rk_ctx* c, uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real);
// the indicator's and the Chebyshev comparator's coefficients the circuits use (circuits.cpp)
const std::vector<double>& indicator_coeffs_of(rk_ctx* c, uint32_t N);
const std::vector<double>& comparator_coeffs_of(rk_ctx* c);

// host number theory (context.cu)
u64 h_mulmod(u64 a, u64 b, u64 q);
u64 h_powmod(u64 a, u64 e, u64 q);
u64 h_invmod(u64 a, u64 q);
int64_t round_half_away(double x);
