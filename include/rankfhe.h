/*
 * rankfhe - encrypted ranking, order statistics and sorting under RNS-CKKS on
 * NVIDIA GB300 (sm_103a).  C ABI.
 *
 * The method is that of "Efficient Ranking, Order Statistics, and Sorting under
 * CKKS" (Mazzone, Everts, Hahn, Peter; arxiv 2412.15126): all N x N pairwise
 * comparisons of an encrypted vector are packed into the slots of one
 * ciphertext by the ReplR / ReplC / TransR re-encoding (Sec. 2.3, Alg. 1, 10,
 * 11), a composite sign polynomial gives the comparison matrix (Sec. 2.2), SumR
 * gives the ranks (Alg. 3, Alg. 8) and the tie-correction offset makes them a
 * permutation (Alg. 6).
 *
 * Conventions for every function:
 *  - Return RK_OK on success; on failure a non-zero rk_status and a thread-local
 *    message readable with rk_last_error().  No C++ exception crosses the ABI.
 *  - Inputs are borrowed and never modified.  Every rk_ct* written through an
 *    output argument is owned by the caller and released with rk_ct_free().
 *  - Device work is ordered on the context's CUDA stream.  Functions that return
 *    host-visible data (decrypt, export, moduli) synchronise that stream.
 *  - A context is used by one host thread at a time.
 *  - Ciphertexts live in device memory in the evaluation (NTT) domain as
 *    64-bit residues, limb-major: [2][L+1][n] words, limbs 0..level in use.
 *  - Canonical exchange form (import/export): coefficient domain, residues in
 *    [0, q), little-endian uint64, layout [2][level+1][n] for a ciphertext.
 */
#ifndef RANKFHE_H
#define RANKFHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rk_ctx rk_ctx;
typedef struct rk_ct rk_ct;

typedef enum {
    RK_OK = 0,
    RK_EINVAL = 1,    /* bad argument (size, range, layout, level mismatch)            */
    RK_ENOMEM = 2,    /* device or host allocation failed                               */
    RK_EDEPTH = 3,    /* the circuit needs more levels than the ciphertext has left     */
    RK_ETIMEOUT = 4,  /* reserved: no kernel here waits on a flag or peer (finite grids) */
    RK_ECUDA = 5,     /* a CUDA runtime call failed (message has the CUDA error text)   */
    RK_EFORMAT = 6,   /* malformed or truncated serialised data                         */
    RK_ENOKEY = 7     /* a switching key (relinearisation or rotation) is missing      */
} rk_status;

/* Parameter set.  Moduli are derived deterministically from these sizes:
 * q_0 = largest prime < 2^log_q0 with q = 1 mod 2n; q_L..q_1 chosen top down,
 * q_l the unused prime = 1 mod 2n nearest floor(Delta_l^2 / 2^log_scale) (ties to
 * the smaller) with Delta_L = 2^log_scale and Delta_{l-1} = Delta_l^2 / q_l;
 * the n_special special primes are the largest unused primes < 2^log_special. */
typedef struct {
    uint32_t log_n;        /* ring degree n = 2^log_n (Sec. 2.1), 10..17                 */
    uint32_t n_limbs;      /* number of primes in Q (L + 1)                              */
    uint32_t n_special;    /* number of special primes alpha (hybrid key switching)      */
    uint32_t digit_size;   /* limbs per key-switching digit                              */
    uint32_t log_scale;    /* log2 of the top-level scale Delta_L                        */
    uint32_t log_q0;       /* bit bound of q_0                                           */
    uint32_t log_special;  /* bit bound of the special primes (<= 61)                    */
    uint32_t d_g;          /* compositions of g in Cmp (Sec. 2.2)                         */
    uint32_t d_f;          /* compositions of f in Cmp (Sec. 2.2)                         */
    uint32_t cmp_cheb;     /* 0: the composite f/g comparison; else the Chebyshev-
                              approximated comparison (Sec. 2.2) with this many
                              coefficients (a power of two, 4..16384): the interpolant at
                              first-kind nodes on [-1, 1] of the step 1 / 1/2 / 0, odd part
                              plus 1/2, by Paterson-Stockmeyer; depth log2(count) + 1      */
    uint32_t prime_form;   /* 0: every prime = 1 mod 2n (as above); 1: every prime = 1 mod
                              2^32, i.e. k 2^32 + 1, by the same rules with 2^32 in place
                              of 2n (the kernels then multiply by q with one 32-bit
                              product; results are the same words for the same primes).
                              Needs log_scale, log_q0, log_special >= 34; at scales near
                              2^45 the chosen primes lie within a few percent of the
                              scale and the canonical scales absorb the spread          */
} rk_params;

/* Ciphertext slot layouts (Sec. 2.3 row-by-row encoding; slot q*N^2 + i*N + j is
 * row i, column j of packed query q). */
#define RK_LAYOUT_ROW 0u   /* vector in row 0: slots q*N^2 + j            */
#define RK_LAYOUT_COL 1u   /* vector in column 0: slots q*N^2 + i*N       */

/* Plaintext mask kinds (Sec. 2.3 MaskR/MaskC, Alg. 6, padding of Sec. 3.1). */
#define RK_MASK_ROW0  1u   /* 1 on row 0 of each N x N block                           */
#define RK_MASK_COL0  2u   /* 1 on column 0 of each block                              */
#define RK_MASK_TIE   3u   /* 4*[j >= i] - 2 on each block (folded Alg. 6)             */
#define RK_MASK_TRI   4u   /* [j >= i] on each block (Alg. 6 delta mask)               */
#define RK_MASK_VALID 5u   /* 1 on rows and columns < n_real of each block (padding)   */
#define RK_MASK_ROW0S 6u   /* 1/D on row 0 (MaskR that also divides ranks by D); D is the
                              n_real argument where one is given, else N              */
#define RK_MASK_COL0S 7u   /* 1/D on column 0 (D as for RK_MASK_ROW0S)                 */
#define RK_MASK_TIEC  8u   /* 4*[j <= i] - 2: column form of RK_MASK_TIE               */
#define RK_MASK_SORTIDX 9u /* -(j+1)/N at row i, column j (Alg. 5 index constant / N)  */
#define RK_MASK_ROWIDX 10u /* -(i+1)/D at row i (Alg. 8 offset less its block constant;
                              D = n_real where given, else N)                          */

/* Key kinds for rk_key_import. */
#define RK_KEY_RELIN  1u
#define RK_KEY_GALOIS 2u

/* Flags for rk_rank. */
#define RK_TIES_CORRECT 1u /* add the tie-correction offset (Alg. 6): ranks become a permutation */
/* Flags for rk_order_stat. */
#define RK_TIES_FIRST 0u   /* tie-corrected ranks: one-hot at the first (lowest index) of equal elements */
#define RK_TIES_ALL   2u   /* k = 1 / k = N: mark every minimum / maximum (Cmp_G / Cmp_GE, Sec. 3.2) */

/* ---- context -------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (e.g. a PyTorch stream's handle) or NULL for a stream owned by the context.
 * Builds the prime chain, NTT twiddle tables and basis-conversion constants.
 * Errors: RK_EINVAL for out-of-range sizes, RK_ECUDA, RK_ENOMEM. */
rk_status rk_ctx_create(const rk_params* params, int device, void* cuda_stream, rk_ctx** out);
void rk_ctx_destroy(rk_ctx* ctx);

/* The prime chain and canonical scales a parameter set gives (the rules above), on
 * the host, without a device or a context: moduli (may be NULL) receives min(cap,
 * L+1+alpha) words, q_0..q_L then p_0..p_{alpha-1}; *count (may be NULL) the number
 * of moduli; scales (may be NULL) min(scales_cap, L+1) doubles Delta_0..Delta_L.
 * The same values rk_ctx_moduli and rk_ctx_scales return for a context of these
 * parameters.  Errors: RK_EINVAL on NULL params or parameters rk_ctx_create rejects. */
rk_status rk_params_chain(const rk_params* params, uint64_t* moduli, size_t cap, size_t* count, double* scales,
                          size_t scales_cap);

/* The moduli q_0..q_L followed by p_0..p_{alpha-1}; *count receives L+1+alpha.
 * Writes min(cap, count) words.  Errors: RK_EINVAL on NULL. */
rk_status rk_ctx_moduli(const rk_ctx* ctx, uint64_t* out, size_t cap, size_t* count);
/* The canonical scales Delta_0..Delta_L (doubles); writes min(cap, L+1). */
rk_status rk_ctx_scales(const rk_ctx* ctx, double* out, size_t cap);
/* Block until all work queued on the context stream has finished. */
rk_status rk_sync(rk_ctx* ctx);
/* Counters since creation: [key switches, rotations, ciphertext products, rescales]. */
rk_status rk_ctx_counters(const rk_ctx* ctx, uint64_t out[4]);

/* Execution options (the paper has no counterpart; results do not depend on them,
 * except RK_OPT_TRIM_LEVELS, which changes the output level).
 * RK_OPT_KS_FUSED: 0 (default) runs hybrid key switching as staged kernels, which
 *   materialise every lifted digit in device memory; 1 fuses the ModUp and ModDown
 *   conversions into the NTT column passes and the key inner product and the final
 *   combine into the row passes (fewer device-memory passes, less parallelism:
 *   slower on GB300 at n = 2^16).  Both produce identical ciphertexts bit for bit.
 * RK_OPT_KS_GROUP_BYTES: bytes of lifted digits the fused path keeps in flight
 *   between its column and row kernels (default 48 MiB, sized for the 129 MB L2);
 *   values below one limb group run one target limb at a time.
 * RK_OPT_BLOCK_STACKING: 1 (default) runs the blocks and block pairs of
 *   rk_rank_blocked (flags 0) as stacks; 0 runs every block and pair ciphertext with
 *   its own launches (the plain per-query form, for comparison).  Same results.
 * RK_OPT_PAIR_PACKING: 1 (default) lets the blocked circuits (rk_rank_blocked,
 *   rk_order_stat_blocked, rk_sort_blocked and rk_rank_blocked_partial) pack their
 *   block-pair work into the free tiles of a ciphertext: a block of B values fills
 *   Q B^2 of the n/2 slots, so up to T = (n/2)/(Q B^2) comparisons (and, for the
 *   blocked order statistic and sort, indicators) run as one ciphertext, moved in and
 *   out by trees of rotations by +-Q B^2 2^s.  It applies when T >= 2, block stacking
 *   is on and the keys of those rotations exist (rk_keygen makes all of them for
 *   B <= max_len / 2 and all but +-n/4 otherwise); the ciphertexts then carry the
 *   packing rotations' noise (same decryption within the circuits' tolerance).  0 runs
 *   every pair on its own ciphertext.
 * RK_OPT_STACK_BUDGET: bytes of device memory one stacked step of the blocked circuits
 *   may take (default 16 GiB): the forms of the blocks and the block-pair comparisons
 *   run in chunks of whole packing groups that fit it, so L is bounded by memory for
 *   the L output blocks only.  RK_OPT_INDICATOR_BUDGET: the same for the blocked order
 *   statistic's and sort's indicator evaluations (default 4 GiB).  Results never
 *   depend on either.
 * RK_OPT_MODUP_COL: 1 runs the staged path's ModUp conversion inside the forward
 *   NTT's column pass (one kernel, the lifted digits written once, in the pass's
 *   output form); 0 (default) converts, then transforms.  rk_autotune picks one.
 *   Results never depend on it.
 * RK_OPT_NTT_GROUP_BYTES: a forward or inverse NTT of more bytes runs as groups of
 *   limbs of at most this size, both passes of a group before the next (0: one launch
 *   pair for the whole set; rk_autotune picks a size).  Results never depend on it.
 * RK_OPT_SERVER_LANES: execution lanes of the next rk_server_start (1 to 16, default 2):
 *   each runs its own batch on its own stream, so batches overlap on the device.
 * RK_OPT_TRIM_LEVELS: 0 (default) evaluates rk_rank / rk_rank_batch at the input's
 *   level; 1 first brings the input down (scalar products by 1 and rescales, as
 *   rk_level_down) to the lowest level the rank circuit needs, so that every key
 *   switch runs on fewer limbs; the result leaves at the lowest level whose modulus
 *   holds ranks up to N at its scale with two bits to spare (level 0 when q_0 has
 *   room, e.g. a 60-bit q_0 at scale 2^45).  The ranks are the same up to rounding;
 *   the ciphertexts differ.
 * Errors: RK_EINVAL for an unknown option or a negative value. */
#define RK_OPT_KS_FUSED 1
#define RK_OPT_KS_GROUP_BYTES 2
#define RK_OPT_BLOCK_STACKING 3
#define RK_OPT_TRIM_LEVELS 4
#define RK_OPT_SERVER_LANES 5
#define RK_OPT_PAIR_PACKING 6
#define RK_OPT_STACK_BUDGET 7
#define RK_OPT_INDICATOR_BUDGET 8
#define RK_OPT_NTT_GROUP_BYTES 9
#define RK_OPT_MODUP_COL 10
rk_status rk_ctx_set_option(rk_ctx* ctx, uint32_t option, int64_t value);

/* Autotune the launch shapes on this device (the paper has no counterpart): times
 * every candidate block width of the four NTT passes for large (224 limbs) and small
 * (2 x 3 limbs) limb sets; the forward NTT of a top-level ModUp set in one launch pair
 * and in limb groups of at most 96, 64 and 32 MiB (both passes of a group before the
 * next, so the data between the passes stays in L2); and, when a rotation key exists,
 * one top-level rotation with staged and with fused key switching (three L2 group
 * sizes).  Keeps the fastest of each.  Results never depend on the choice.  report
 * (may be NULL) receives, for the NTT slots [small][inverse][column] in that nesting
 * order, (width, us) pairs (16 values), then the four group timings in us and the
 * chosen group MiB (0: whole set), then, with a rotation key, staged us, fused us at
 * 24/48/96 MiB and the choice (0 staged, else the group MiB), then the staged path
 * with the ModUp conversion in the column pass (us) and whether it was chosen (1/0);
 * *count receives the number of values. */
rk_status rk_autotune(rk_ctx* ctx, double* report, size_t cap, size_t* count);

/* ---- keys ----------------------------------------------------------------- */

/* Generate secret, public, relinearisation key and the rotation (Galois) keys
 * the circuits need for every power-of-two length N <= max_len (Sec. 3.1: the
 * rotations of ReplR, ReplC, TransR, SumR, SumC, TransC), on the device, from
 * `seed` (SplitMix64 counter stream).  The switching keys are seeded (see
 * rk_key_import_seeded): only their b parts are stored.
 * Errors: RK_EINVAL, RK_ENOMEM, RK_ECUDA. */
rk_status rk_keygen(rk_ctx* ctx, uint64_t seed, uint32_t max_len);

/* Add rotation keys for left rotations by r[i] slots (negative = right). */
rk_status rk_keygen_rotations(rk_ctx* ctx, const int32_t* r, size_t count);

/* Import a ternary secret s (n signed coefficients in {-1,0,1}). */
rk_status rk_secret_import(rk_ctx* ctx, const int64_t* s, size_t n);

/* Import a switching key made elsewhere (e.g. by a reference implementation).
 * kind: RK_KEY_RELIN (galois ignored) or RK_KEY_GALOIS with its Galois element.
 * coeffs: [beta_L][2][L+1+alpha][n] words, coefficient domain, residues in
 * [0, q) in prime order q_0..q_L, p_0..p_{alpha-1}; entry [j][0] is b_j, [j][1]
 * is a_j with b_j = -a_j s + e_j + P E_j s' (E_j the CRT idempotent of digit j).
 * Errors: RK_EINVAL if words does not match, RK_ENOMEM. */
rk_status rk_key_import(rk_ctx* ctx, uint32_t kind, uint64_t galois, const uint64_t* coeffs, size_t words);

/* Import a seeded switching key: coeffs = [beta_L][L+1+alpha][n] words, the b_j
 * parts only (coefficient domain, residues in [0, q)); every a_j is regenerated from
 * `seed` by the key switch itself.  For digit j, prime index p (q_0..q_L, then
 * p_0..p_{alpha-1}) and evaluation index i (the value at psi^(2 brev(i) + 1)), let x
 * be element c = (j (L+1+alpha) + p) n + i of the SplitMix64 stream from `seed`
 * (x = mix(seed + (c + 1) 0x9E3779B97F4A7C15), the generator's published
 * definition); the high 64 bits of x q_p are a_j's evaluation there times 2^64,
 * mod q_p.  Seeded keys halve key memory and the key switch's key traffic;
 * rk_keygen makes them.  Errors: RK_EINVAL if words does not match, RK_EFORMAT,
 * RK_ENOMEM. */
rk_status rk_key_import_seeded(rk_ctx* ctx, uint32_t kind, uint64_t galois, uint64_t seed, const uint64_t* coeffs,
                               size_t words);

/* Every switching key of the context (relinearisation, then Galois keys by element)
 * as one blob of little-endian 64-bit words: magic "RKKEYS02", log_n, L+1+alpha,
 * beta_L, the key count K, then K records [kind][galois][seeded][seed][words][words
 * of rk_key_import's layout, or of rk_key_import_seeded's when seeded is 1].
 * buf NULL: *len receives the size only; otherwise buf
 * (8-byte aligned, cap >= *len bytes) receives the blob.  The secret is not included.
 * Errors: RK_EINVAL (buffer too small or unaligned), RK_ECUDA. */
rk_status rk_keys_export(rk_ctx* ctx, uint8_t* buf, size_t cap, size_t* len);
/* Import every key of a blob from rk_keys_export (parameters must match).
 * Errors: RK_EFORMAT (bad magic, parameters, length), RK_EINVAL, RK_ENOMEM. */
rk_status rk_keys_import(rk_ctx* ctx, const uint8_t* buf, size_t len);

/* Galois element of a left rotation by r slots: 5^r mod 2n. */
uint64_t rk_galois_left(const rk_ctx* ctx, int32_t r);

/* ---- encoding ---------------------------------------------------------------- */

/* Override the unscaled encoding (n doubles: the real polynomial whose slot
 * values are the mask) used for mask `kind` at (N, Q, n_real).  By default the
 * library computes it with its own FFT; importing a table from another
 * implementation makes plaintext products bit-identical to it.
 * Errors: RK_EINVAL on a bad kind or length. */
rk_status rk_encoding_import(rk_ctx* ctx, uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real,
                             const double* u, size_t n);

/* The unscaled encoding the library uses for mask `kind` at (N, Q, n_real): n doubles,
 * the real polynomial whose slot values are the mask (Sec. 2.1 canonical embedding:
 * slot j <-> zeta^(5^j)), from the library's own FFT unless rk_encoding_import replaced
 * it.  u receives n values.  Errors: RK_EINVAL on a bad kind, shape or length. */
rk_status rk_encoding_export(rk_ctx* ctx, uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real, double* u, size_t n);

/* The Chebyshev coefficients of the indicator window the order-statistic and sorting
 * circuits use for padded length N (Alg. 4, 5; see rk_indicator_import), computed by
 * the library unless imported.  *count receives their number; out (may be NULL)
 * receives min(cap, count) values.  Errors: RK_EINVAL. */
rk_status rk_indicator_export(rk_ctx* ctx, uint32_t N, double* out, size_t cap, size_t* count);

/* The Chebyshev comparator's coefficients (Sec. 2.2; the context's cmp_cheb of them),
 * computed by the library unless imported; out and count as rk_indicator_export.
 * Errors: RK_EINVAL if the context uses the composite comparator. */
rk_status rk_comparator_export(rk_ctx* ctx, double* out, size_t cap, size_t* count);

/* Override the Chebyshev coefficients c_0..c_{count-1} of the indicator window
 * used for vectors of padded length N (Alg. 4, 5: Ind_k(r) = p((r - k)/N) with
 * p = sum_i c_i T_i).  By default the library interpolates sinc^2(N t) at the
 * count = max(8N, 128) Chebyshev nodes of the first kind with its own transform.  count
 * must be a power of two >= 4.  Errors: RK_EINVAL. */
/* Replace the Chebyshev comparator's coefficients (cmp_cheb of them) with another
 * implementation's, so that results can be compared bit for bit.
 * Errors: RK_EINVAL if the context does not use the Chebyshev comparator or the count
 * differs. */
rk_status rk_comparator_import(rk_ctx* ctx, const double* coeffs, size_t count);

rk_status rk_indicator_import(rk_ctx* ctx, uint32_t N, const double* coeffs, size_t count);

/* ---- client operations ------------------------------------------------------ */

/* Encode and encrypt (public key) `count` values into row 0 of packed queries:
 * value i goes to query i / n_real, column i % n_real.  N is the padded length
 * (a power of two >= n_real with Q*N*N <= n/2), Q the number of packed queries.
 * Values must lie in [0, 1) (the comparator's domain, Sec. 2.2): else RK_EINVAL. */
rk_status rk_encrypt(rk_ctx* ctx, const double* v, uint32_t count, uint32_t N, uint32_t Q,
                     uint32_t n_real, rk_ct** out);

/* Decrypt and decode all n/2 slots (real parts) into out[0..cap). */
rk_status rk_decrypt_slots(rk_ctx* ctx, const rk_ct* ct, double* out, size_t cap);

/* Decrypt the result vector: row 0 (or column 0 for RK_LAYOUT_COL) of each packed
 * query, n_real values per query, Q*n_real values written when cap allows.
 * *n_out receives Q*n_real. */
rk_status rk_decrypt(rk_ctx* ctx, const rk_ct* ct, double* out, size_t cap, uint32_t* n_out);

/* Import a ciphertext in canonical form ([2][level+1][n] coefficient-domain
 * residues) with its vector metadata.  Errors: RK_EINVAL. */
rk_status rk_ct_import(rk_ctx* ctx, const uint64_t* coeffs, uint32_t level, uint32_t N, uint32_t Q,
                       uint32_t n_real, rk_ct** out);
/* Stack `count` ciphertexts of the same level and vector shape into one handle
 * ([count][2][L+1][n] in device memory, copied): every operation and circuit on a
 * stacked handle runs all of them with one launch per kernel, each switching key
 * read once per 8 ciphertexts.  Errors: RK_EINVAL on a shape mismatch. */
rk_status rk_ct_stack(rk_ctx* ctx, const rk_ct* const* in, uint32_t count, rk_ct** out);
/* Split a stacked handle into rk_ct_count(in) single ciphertexts (copied). */
rk_status rk_ct_unstack(rk_ctx* ctx, const rk_ct* in, rk_ct** outs);
/* Number of ciphertexts in a handle (1 unless stacked). */
uint32_t rk_ct_count(const rk_ct* ct);

/* Export in canonical form; cap in words must be >= 2*(level+1)*n. */
rk_status rk_ct_export(const rk_ct* ct, uint64_t* coeffs, size_t cap);
uint32_t rk_ct_level(const rk_ct* ct);
void rk_ct_free(rk_ct* ct);

/* ---- homomorphic operations (Sec. 2.1) --------------------------------------- */

/* Left rotation by r slots (r < 0: right rotation by -r): slot s <- slot s + r.
 * The automorphism X -> X^(5^r) is applied to the lifted digits of the key switch.
 * Errors: RK_ENOKEY if the rotation key is missing. */
rk_status rk_rotate(rk_ctx* ctx, const rk_ct* in, int32_t r, rk_ct** out);
/* Several rotations of one ciphertext sharing one ModUp (hoisting). */
rk_status rk_rotate_many(rk_ctx* ctx, const rk_ct* in, const int32_t* r, uint32_t k, rk_ct** outs);
rk_status rk_add(rk_ctx* ctx, const rk_ct* a, const rk_ct* b, rk_ct** out);
rk_status rk_sub(rk_ctx* ctx, const rk_ct* a, const rk_ct* b, rk_ct** out);
/* Add the constant v to every slot (v * Delta_level rounded half away from zero). */
rk_status rk_add_const(rk_ctx* ctx, const rk_ct* a, double v, rk_ct** out);
/* Product with relinearisation and rescale: out at level-1. */
rk_status rk_mul(rk_ctx* ctx, const rk_ct* a, const rk_ct* b, rk_ct** out);
/* Product with the constant v, rescaled: out at level-1. */
rk_status rk_mul_scalar(rk_ctx* ctx, const rk_ct* a, double v, rk_ct** out);
/* Product with a mask plaintext (RK_MASK_*), rescaled: out at level-1. */
rk_status rk_mul_mask(rk_ctx* ctx, const rk_ct* a, uint32_t kind, rk_ct** out);
/* Drop one prime by rounding division (rescale); out at level-1, scale divided by q_level. */
rk_status rk_rescale(rk_ctx* ctx, const rk_ct* a, rk_ct** out);

/* Rescale without any device allocation, for callers that cannot allocate device
 * memory on the call path (e.g. where another runtime has reserved the device
 * memory in its own pool, or in a loop that must never enter the CUDA allocator).
 * The paper has no counterpart; it is rk_rescale on caller-owned buffers.
 * d_in:  device buffer [2][level+1][n] words, evaluation domain (the layout of
 *        rk_ntt_forward applied to each polynomial of a canonical ciphertext);
 * d_out: device buffer [2][level][n] words, receives the rescaled ciphertext in
 *        the same domain; it must not overlap d_in.
 * The temporary lives in one fixed 4 MiB array in device memory declared by the
 * library (held by every GPU that loads the library until the process exits), so
 * 2*(level+1)*n must not exceed 2^19 words: larger sizes fail with RK_EINVAL.
 * The first call on each context resolves that array's address (with the context's
 * device current) and keeps it in the context; make that first call before any CUDA
 * stream capture.  A context created after the device was reset resolves it anew; a
 * context that outlives a reset of its device is unusable, as for every call.  All
 * calls share the array (nothing in it needs to start at zero): calls whose work
 * overlaps on the GPU, e.g. from two contexts on different streams of one device,
 * race.  Work is queued on the context stream.  rk_device_alloc_count() does not
 * change across a call.
 * Errors: RK_EINVAL (NULL, level out of range, too large, overlap), RK_ECUDA. */
rk_status rk_rescale_noalloc(rk_ctx* ctx, const uint64_t* d_in, uint64_t* d_out, uint32_t level);

/* ---- circuits (Sec. 3-4) ------------------------------------------------------ */

/* Rank (Alg. 3): fractional ranks of the vector in row 0 of `in` (fresh, top
 * level), in row 0 of the output.  flags: RK_TIES_CORRECT adds the tie-correction
 * offset of Alg. 6.  The circuit takes 2 + the comparison's levels (+1 for a padded
 * vector, +2 with RK_TIES_CORRECT); with RK_OPT_TRIM_LEVELS the input is first
 * brought down to that many levels plus the level the result must keep.
 * Errors: RK_EDEPTH if the parameters lack the levels, RK_ENOKEY, RK_EINVAL. */
rk_status rk_rank(rk_ctx* ctx, const rk_ct* in, uint32_t flags, rk_ct** out);

/* Comparison matrix (Alg. 3 lines 1-3): C = Cmp(ReplR(V), ReplC(TransR(V))), slot
 * q*N^2 + i*N + j holding Cmp(v_j, v_i) of Eq. 1 approximated by the composite
 * (f^d_f o g^d_g)(x)/2 + 1/2 of Sec. 2.2.  Errors as rk_rank. */
rk_status rk_compare_matrix(rk_ctx* ctx, const rk_ct* in, rk_ct** out);

/* k-th order statistic (Alg. 4): a 0/1 row marking the element(s) of rank k
 * (1 <= k <= N; k = 1 argmin, k = N argmax), Ind_k evaluated by Paterson-Stockmeyer
 * in the Chebyshev basis.  flags: RK_TIES_FIRST (tie-corrected ranks, one-hot at
 * the first of equal elements) or RK_TIES_ALL (k = 1 or N: every minimum / maximum;
 * other k: fractional ranks).  Errors: RK_EDEPTH, RK_ENOKEY, RK_EINVAL. */
rk_status rk_order_stat(rk_ctx* ctx, const rk_ct* in, uint32_t k, uint32_t flags, rk_ct** out);

/* Value of the k-th smallest element (Alg. 4 with the value retrieval of Sec. 3.2):
 * SumC(O . V) with O the tie-corrected one-hot mask of rank k, so the division by the
 * mask's L1 norm is by one.  The value is in slot 0 of each query block (column 0 of
 * row 0); the other slots of row 0 are zero.  Errors as rk_order_stat. */
rk_status rk_order_value(rk_ctx* ctx, const rk_ct* in, uint32_t k, rk_ct** out);

/* Value of the k-th order statistic from the all-ties mask (Sec. 3.2): O = the
 * rk_order_stat mask with RK_TIES_ALL (k = 1: every minimum, k = N: every maximum,
 * other k: the elements of fractional rank k), and the value <O, V> / |O|_1 =
 * SumC(O . V) / SumC(O), the division by Goldschmidt's iteration on SumC(O) / N
 * (d iterations, d the smallest with (1 - 1/N)^(2^(d+1)) <= 2^-10: 5 at N = 8, 9 at
 * N = 128).  The value is in slot 0 of each query block, zero if no element has rank
 * k.  Takes the order statistic's levels plus d + 4.
 * Errors: RK_EDEPTH, RK_ENOKEY, RK_EINVAL. */
rk_status rk_order_value_all(rk_ctx* ctx, const rk_ct* in, uint32_t k, rk_ct** out);

/* Median (Alg. 4's particular case): the (N+1)/2-th smallest value for odd N, the mean
 * of the N/2-th and (N/2+1)-th for even N, from one tie-corrected rank; in slot 0 as
 * for rk_order_value.  Errors as rk_order_stat. */
rk_status rk_median(rk_ctx* ctx, const rk_ct* in, rk_ct** out);

/* Sort (Alg. 5, column form of Sec. 3.3, with the tie-correction offset of Alg. 6):
 * the ascending values in row 0 of the output.  Errors as rk_order_stat. */
rk_status rk_sort(rk_ctx* ctx, const rk_ct* in, uint32_t flags, rk_ct** out);

/* Multi-ciphertext ranking (Alg. 7, Sec. 5): a vector of L*B values split into L
 * blocks of B (a power of two with B^2 <= n/2), block i encrypted in row 0 of
 * blocks[i] (all at one level, unpadded).  outs[i] receives the fractional ranks of
 * block i's values among all L*B values, in row 0.  Only the L(L+1)/2 comparisons
 * C_{i,j}, j >= i, are evaluated (Eq. 3), as one stacked circuit.  flags: 0, or
 * RK_TIES_CORRECT for the stable ranks (Alg. 6 across blocks: equal values count
 * when they sit in an earlier block or at an earlier position of the same block;
 * per block pair, the diagonal pair takes the folded offset, the others
 * Cmp_G = 2C^2 - C or its complement).  Errors: RK_EDEPTH, RK_ENOKEY, RK_EINVAL. */
rk_status rk_rank_blocked(rk_ctx* ctx, const rk_ct* const* blocks, uint32_t L, uint32_t flags, rk_ct** outs);

/* rk_rank_blocked (flags 0) in two parts, so that the L(L+1)/2 block comparisons (the
 * parallel loop over block pairs of Sec. 5) can be divided between devices and only
 * their partial sums exchanged.  Part one evaluates C_{i,j} = Cmp(ReplR(V_i),
 * ReplC(TransR(V_j))) for the npairs listed pairs (pair_i[p] <= pair_j[p] < L) and
 * writes, per block i, A[i] = the sum of the listed C_{i,j} and B[i] = the sum of the
 * listed C_{j,i} with j < i (an encryption of zero with no noise where no listed pair
 * contributes), all at the comparison's output level.  Part two takes the sums over
 * all parts (rk_add of the parts' A[i], and of their B[i]) and returns
 * outs[i] = TransC(SumC(i - B[i])) + SumR(A[i]) + 1/2 (Eq. 3), bit-identical to
 * rk_rank_blocked when the parts together list every pair once.  Blocks as for
 * rk_rank_blocked; every output is owned by the caller.
 * Errors: RK_EINVAL (a pair out of range, mismatched sums), RK_EDEPTH, RK_ENOKEY. */
rk_status rk_rank_blocked_partial(rk_ctx* ctx, const rk_ct* const* blocks, uint32_t L, const uint32_t* pair_i,
                                  const uint32_t* pair_j, uint32_t npairs, rk_ct** A, rk_ct** B);
rk_status rk_rank_blocked_finish(rk_ctx* ctx, const rk_ct* const* A, const rk_ct* const* B, uint32_t L, rk_ct** outs);

/* Order statistic over a multi-ciphertext vector (Alg. 4 on the tie-corrected
 * blocked ranks of rk_rank_blocked): outs[i] marks, in row 0, the element of block i
 * whose stable rank is k (1 <= k <= L*B), one-hot over the whole vector.  The
 * indicator is the sinc^2 window for the length L*B.  flags must be RK_TIES_FIRST.
 * Errors as rk_rank_blocked. */
rk_status rk_order_stat_blocked(rk_ctx* ctx, const rk_ct* const* blocks, uint32_t L, uint32_t k, uint32_t flags,
                                rk_ct** outs);

/* Multi-ciphertext sorting (Alg. 8) on the tie-corrected blocked ranks: outs[i]
 * holds, in row 0, the values of ranks B i + 1 .. B (i + 1) in ascending order.
 * The L^2 indicators run as stacked circuits, in chunks that bound the working
 * set.  flags must be 0.  Errors as rk_rank_blocked. */
rk_status rk_sort_blocked(rk_ctx* ctx, const rk_ct* const* blocks, uint32_t L, uint32_t flags, rk_ct** outs);

/* Ranks of `count` ciphertexts (each its own query set).  Inputs of the same level
 * and vector shape are stacked and run as one circuit (one launch per kernel for
 * the group); out[i] is the rank ciphertext of in[i]. */
rk_status rk_rank_batch(rk_ctx* ctx, const rk_ct* const* in, size_t count, uint32_t flags, rk_ct** out);
/* The same grouping for order statistics (one k for all) and sorts. */
rk_status rk_order_stat_batch(rk_ctx* ctx, const rk_ct* const* in, size_t count, uint32_t k, uint32_t flags, rk_ct** out);
rk_status rk_sort_batch(rk_ctx* ctx, const rk_ct* const* in, size_t count, uint32_t flags, rk_ct** out);

/* ---- serving loop ------------------------------------------------------------ */

/* Serving loop with continuous batching (the paper has no serving layer; this is the
 * batched form of Alg. 3-5 and 7 under a request stream).  The server runs
 * RK_OPT_SERVER_LANES execution lanes, each a worker thread with its own stream,
 * key-switching scratch (sized for stacks of 16 at start) and plaintext caches over
 * the context's keys, so that batches on different lanes overlap on the device.
 * Requests are queued from any thread.  Whenever a lane is free and the running
 * batches leave room in `mem_budget_bytes` for the oldest queued request (a lane with
 * nothing else running always takes it), the lane takes that request and every
 * queued request of the same operation, arguments and ciphertext shape (level, N, Q,
 * n_real, layout), up to `max_stack` ciphertexts and the room left, and evaluates
 * them as one stacked circuit.  Single-ciphertext requests of padded length N with
 * Q = (n/2)/N^2 >= 2 are slot-packed first when the packing rotations' keys exist
 * (left rotations by +-N^2 2^k, 2^k < Q; rk_keygen makes all of them except +-n/4,
 * which rk_keygen_rotations adds): up to Q requests share a ciphertext (Sec. 2.3
 * layout), packed and unpacked by trees of stacked rotations.  Results of unpacked
 * requests are bit-identical to the request alone; packed results carry the packing
 * rotations' noise and decrypt to the request's values alone within the circuit's
 * tolerance (other slots hold other requests' results).
 * While a server runs, it owns the context: other threads may call only rk_server_*
 * and rk_ct_free on collected results until rk_server_stop returns.  Inputs are
 * borrowed: keep each submitted ciphertext alive and unchanged until its result has
 * been collected.  Results are owned by the caller once collected. */
#define RK_OP_RANK 1          /* rk_rank(in, flags) */
#define RK_OP_ORDER_STAT 2    /* rk_order_stat(in, arg = k, flags) */
#define RK_OP_SORT 3          /* rk_sort(in, flags) */
#define RK_OP_RANK_BLOCKED 4  /* rk_rank_blocked(blocks of a stack (rk_ct_stack), flags);
                                 the result is the stack of the rank blocks */
#define RK_OP_ORDER_STAT_BLOCKED 5   /* rk_order_stat_blocked(blocks of a stack, arg = k) */
#define RK_OP_SORT_BLOCKED 6  /* rk_sort_blocked(blocks of a stack) */
rk_status rk_server_start(rk_ctx* ctx, size_t mem_budget_bytes, uint32_t max_stack);
/* Queue a request; *ticket identifies it.  Errors: RK_EINVAL (no server, unknown op,
 * a stack where one ciphertext is expected, server stopping). */
rk_status rk_server_submit(rk_ctx* ctx, uint32_t op, uint32_t arg, uint32_t flags, const rk_ct* in, uint64_t* ticket);
/* Collect a finished request: *out = its result, or NULL while it is pending.  Waits
 * up to timeout_s seconds (0: poll, negative: no limit).  A failed request returns its
 * error status.  Each ticket is collected once; RK_EINVAL for unknown tickets. */
rk_status rk_server_wait(rk_ctx* ctx, uint64_t ticket, double timeout_s, rk_ct** out);
/* rk_server_wait without waiting: *out = the result, or NULL while it is pending. */
rk_status rk_server_poll(rk_ctx* ctx, uint64_t ticket, rk_ct** out);
/* out[8]: requests finished, p50 and p99 and max latency (s, submit to result on the
 * device), batches run, mean batch size, peak device memory in use on the whole device
 * above the level at rk_server_start (bytes; includes other users of the device),
 * requests queued. */
rk_status rk_server_stats(rk_ctx* ctx, double out[8]);
/* out[5]: lanes, most lanes busy at once, mean lanes busy (the batches' run times
 * summed over the span from the first batch's start to the last one's end), requests
 * served slot-packed, scratch bytes of the lanes. */
rk_status rk_server_stats_lanes(rk_ctx* ctx, double out[5]);
/* Latencies (s) of the finished requests in completion order: writes min(cap, count)
 * values; *count receives the number finished. */
rk_status rk_server_latencies(rk_ctx* ctx, double* out, size_t cap, size_t* count);
/* Finish every queued request, stop the worker, free uncollected results. */
rk_status rk_server_stop(rk_ctx* ctx);

/* ---- CUDA graphs -------------------------------------------------------------- */

typedef struct rk_graph rk_graph;

/* Capture the whole rank circuit (rk_rank with `flags`) for inputs shaped like
 * `tmpl` (level, N, Q, n_real, stack size) as one CUDA graph on the context stream.
 * Runs the circuit once first (to build cached plaintexts and size the scratch).
 * Must not be called while the context stream is being captured elsewhere.
 * Errors: as rk_rank, RK_ECUDA if capture or instantiation fails. */
rk_status rk_graph_rank(rk_ctx* ctx, const rk_ct* tmpl, uint32_t flags, rk_graph** out);
/* Capture any circuit as one CUDA graph for inputs shaped like `tmpl` (level, N, Q,
 * n_real, stack size), as rk_graph_rank does for the rank.  op is an RK_OP_* code with
 * the arguments of the serving loop (arg = k for order statistics, flags); for the
 * blocked operations tmpl is a stack of L blocks, block i being members
 * [i B/L, (i+1) B/L) of it (B/L queries a block), and a replay returns the stack of
 * the L output blocks in the same layout.  Errors: as the circuit, RK_EINVAL for an
 * unknown op or L not dividing the stack, RK_ECUDA if capture or instantiation
 * fails. */
rk_status rk_graph_capture(rk_ctx* ctx, uint32_t op, uint32_t arg, uint32_t flags, uint32_t L, const rk_ct* tmpl,
                           rk_graph** out);
/* Replay: copy `in` (same shape as the template) into the captured input, launch
 * the graph and return the result in a new handle (owned by the caller). */
rk_status rk_graph_run(rk_graph* g, const rk_ct* in, rk_ct** out);
void rk_graph_free(rk_graph* g);

/* ---- raw kernels on device buffers (for parity tests and composition) ------- */

/* Forward / inverse negacyclic NTT of `limbs` residue polynomials stored
 * contiguously at device address d_data (limb t uses prime id first_prime + t;
 * prime ids index q_0..q_L, p_0..).  Forward output order: index i holds the
 * evaluation at psi^(2 brev(i) + 1).  Inputs must be in [0, q); outputs are. */
rk_status rk_ntt_forward(rk_ctx* ctx, uint64_t* d_data, uint32_t limbs, uint32_t first_prime);
rk_status rk_ntt_inverse(rk_ctx* ctx, uint64_t* d_data, uint32_t limbs, uint32_t first_prime);

/* ---- measurement ------------------------------------------------------------- */

/* Time every launch of the listed kernel kinds (comma-separated) with CUDA events on
 * the context stream: "ntt_fwd", "ntt_inv", "modup", "ks_inner", "moddown_conv",
 * "ks_combine", "tensor", "rescale", "pointwise", "client"; NULL or "" stops timing.
 * Resets the accumulators.  Errors: RK_EINVAL for an unknown name. */
rk_status rk_profile_start(rk_ctx* ctx, const char* kinds);
/* Synchronise and report the timed launches since rk_profile_start, summed over the
 * kinds: out[0] total milliseconds, out[1] launches (an NTT counts its two passes as
 * one), out[2] algorithmic bytes (each input word read once, each output word written
 * once), out[3] modular products (an NTT: its butterflies).  Stops timing. */
rk_status rk_profile_stop(rk_ctx* ctx, double out[4]);
/* The same four figures for one kind, after rk_profile_stop. */
rk_status rk_profile_kind(const rk_ctx* ctx, const char* kind, double out[4]);
/* Suspend (paused = 1) or resume (0) the timing started by rk_profile_start without
 * synchronising or resetting the accumulators: launches in between are not timed.
 * The events bracketing each timed launch cost a few microseconds of device time
 * (they separate it from its neighbours), so a long run can time a sample of its
 * steps.  Errors: RK_EINVAL on a null context. */
rk_status rk_profile_pause(rk_ctx* ctx, int paused);
/* Integer throughput of the device (the paper has no counterpart): the ceilings of
 * the integer-bound kernels, measured by project-written microbenchmarks with every
 * operand in registers (independent dependency chains per thread, grids over every
 * SM; the best of three timed launches each).  out[0]: 32-bit integer multiply-adds
 * a second; out[1]: 64-bit Shoup modular products a second (x w mod q with a
 * precomputed companion, the NTT's product); out[2]: forward NTT butterflies
 * (Cooley-Tukey, values in [0, 4q)) a second; out[3], out[4]: the Shoup products and
 * butterflies with a prime k 2^32 + 1 and the cheaper product by such a q (the path
 * of contexts whose primes all have that form, prime_form 1).  Synchronises; takes
 * about a second.  Errors: RK_ECUDA. */
rk_status rk_measure_alu(rk_ctx* ctx, double out[5]);
/* Device allocations (cudaMalloc and cudaMallocAsync calls) the library has made in
 * this process, over every context. */
uint64_t rk_device_alloc_count(void);
/* Number of kernels this context has launched since creation. */
uint64_t rk_launch_count(const rk_ctx* ctx);

/* The thread-local message of the last failure on this thread. */
const char* rk_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RANKFHE_H */
