/*
 * Plain CPU oracle: the integer arithmetic of RNS-CKKS (Cheon-Kim-Kim-Song,
 * residue number system variant) that the ranking / order-statistic / sorting
 * circuits of "Efficient Ranking, Order Statistics, and Sorting under CKKS"
 * (Sec. 2.1) run on.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the oracle that the tests,
 * the smoke check and the CPU-baseline leg of the benchmark compare the CUDA
 * path against.  The product path never loads it.  It shares no code, tables
 * or constants with the CUDA library; the one common definition is the
 * published SplitMix64 generator of seeded switching keys, which each side
 * implements on its own from the published description.
 *
 * Everything here is deliberately plain: every modular product is a 128-bit
 * product followed by the C remainder operator, the number-theoretic
 * transform is the textbook iterative radix-2 cyclic transform (used only as
 * a fast way to form the negacyclic ring product, and pinned in the tests to
 * the schoolbook product), and the basis conversion is the formula written
 * out term by term.  OpenMP parallelises over independent residues only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * b) % q);
}
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t s = a + b; /* a, b < q < 2^63: no overflow */
    return s >= q ? s - q : s;
}
static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : a + (q - b);
}
static uint64_t powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}
/* inverse modulo a prime (Fermat) */
static uint64_t invmod(uint64_t a, uint64_t q) { return powmod(a, q - 2, q); }

uint64_t orc_powmod(uint64_t a, uint64_t e, uint64_t q) { return powmod(a, e, q); }
uint64_t orc_invmod(uint64_t a, uint64_t q) { return invmod(a, q); }
uint64_t orc_mulmod(uint64_t a, uint64_t b, uint64_t q) { return mulmod(a, b, q); }

/* Deterministic Miller-Rabin; the first twelve prime bases decide every n < 3.3e24. */
int orc_is_prime(uint64_t n) {
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int k = 1; k < r; k++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* A primitive m-th root of unity modulo prime q (m a power of two dividing q-1):
 * the first candidate c = 2, 3, ... whose power c^((q-1)/m) has order exactly m. */
uint64_t orc_root_of_unity(uint64_t q, uint64_t m) {
    for (uint64_t c = 2;; c++) {
        uint64_t w = powmod(c, (q - 1) / m, q);
        if (powmod(w, m / 2, q) == q - 1) return w;
    }
}

/* Textbook iterative radix-2 cyclic NTT of length n with root w (in place). */
static void ntt_cyclic(uint64_t *a, size_t n, uint64_t w, uint64_t q) {
    for (size_t i = 1, j = 0; i < n; i++) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    uint64_t *tw = (uint64_t *)malloc(sizeof(uint64_t) * (n / 2 + 1));
    for (size_t len = 2; len <= n; len <<= 1) {
        uint64_t wl = powmod(w, n / len, q);
        tw[0] = 1;
        for (size_t k = 1; k < len / 2; k++) tw[k] = mulmod(tw[k - 1], wl, q);
        for (size_t i = 0; i < n; i += len) {
            for (size_t k = 0; k < len / 2; k++) {
                uint64_t u = a[i + k];
                uint64_t v = mulmod(a[i + k + len / 2], tw[k], q);
                a[i + k] = addmod(u, v, q);
                a[i + k + len / 2] = submod(u, v, q);
            }
        }
    }
    free(tw);
}

/* Forward negacyclic transform: a_k <- a_k psi^k, then cyclic NTT with w = psi^2.
 * psi is the primitive 2n-th root chosen by orc_root_of_unity. */
static void nega_forward(uint64_t *a, size_t n, uint64_t q) {
    uint64_t psi = orc_root_of_unity(q, 2 * n);
    uint64_t t = 1;
    for (size_t k = 0; k < n; k++) { a[k] = mulmod(a[k], t, q); t = mulmod(t, psi, q); }
    ntt_cyclic(a, n, mulmod(psi, psi, q), q);
}
static void nega_inverse(uint64_t *a, size_t n, uint64_t q) {
    uint64_t psi = orc_root_of_unity(q, 2 * n);
    uint64_t psi_inv = invmod(psi, q);
    ntt_cyclic(a, n, mulmod(psi_inv, psi_inv, q), q);
    uint64_t n_inv = invmod((uint64_t)(n % q), q);
    uint64_t t = n_inv;
    for (size_t k = 0; k < n; k++) { a[k] = mulmod(a[k], t, q); t = mulmod(t, psi_inv, q); }
}

void orc_nega_forward(uint64_t *a, size_t n, uint64_t q) { nega_forward(a, n, q); }
void orc_nega_inverse(uint64_t *a, size_t n, uint64_t q) { nega_inverse(a, n, q); }

/* Schoolbook product in Z_q[x]/(x^n + 1): x^n = -1 folds the upper half back with a sign. */
void orc_polymul_schoolbook(const uint64_t *a, const uint64_t *b, uint64_t *out, size_t n, uint64_t q) {
    for (size_t k = 0; k < n; k++) out[k] = 0;
    for (size_t i = 0; i < n; i++)
        for (size_t j = 0; j < n; j++) {
            uint64_t p = mulmod(a[i], b[j], q);
            size_t k = i + j;
            if (k < n) out[k] = addmod(out[k], p, q);
            else out[k - n] = submod(out[k - n], p, q);
        }
}

/*
 * Ring products summed over `terms`, residue by residue:
 *   out[l] = sum_t  a[t][l] * b[t][l]   in Z_{q_l}[x]/(x^n+1),  l = 0..limbs-1.
 * a and b are addressed as a + t*a_tstride + l*n (likewise b).  With terms = 1
 * this is the plain ring product of two RNS polynomials.
 */
void orc_ring_mac(const uint64_t *a, size_t a_tstride, const uint64_t *b, size_t b_tstride,
                  int terms, uint64_t *out, int limbs, size_t n, const uint64_t *qs) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int l = 0; l < limbs; l++) {
        uint64_t q = qs[l];
        uint64_t *acc = (uint64_t *)calloc(n, sizeof(uint64_t));
        uint64_t *ta = (uint64_t *)malloc(n * sizeof(uint64_t));
        uint64_t *tb = (uint64_t *)malloc(n * sizeof(uint64_t));
        for (int t = 0; t < terms; t++) {
            memcpy(ta, a + (size_t)t * a_tstride + (size_t)l * n, n * sizeof(uint64_t));
            memcpy(tb, b + (size_t)t * b_tstride + (size_t)l * n, n * sizeof(uint64_t));
            nega_forward(ta, n, q);
            nega_forward(tb, n, q);
            for (size_t k = 0; k < n; k++) acc[k] = addmod(acc[k], mulmod(ta[k], tb[k], q), q);
        }
        nega_inverse(acc, n, q);
        memcpy(out + (size_t)l * n, acc, n * sizeof(uint64_t));
        free(acc); free(ta); free(tb);
    }
}

/* out[l][k] = a[l][k] * c_l mod q_l  (c_l < q_l) */
void orc_mul_scalar(const uint64_t *a, const uint64_t *c, uint64_t *out, int limbs, size_t n, const uint64_t *qs) {
#pragma omp parallel for
    for (int l = 0; l < limbs; l++)
        for (size_t k = 0; k < n; k++)
            out[(size_t)l * n + k] = mulmod(a[(size_t)l * n + k], c[l], qs[l]);
}

/* out[l][k] = a[l][k] * b[l][k] mod q_l (coefficient-wise; used on NTT images and for checks) */
void orc_mul_pointwise(const uint64_t *a, const uint64_t *b, uint64_t *out, int limbs, size_t n, const uint64_t *qs) {
#pragma omp parallel for
    for (int l = 0; l < limbs; l++)
        for (size_t k = 0; k < n; k++)
            out[(size_t)l * n + k] = mulmod(a[(size_t)l * n + k], b[(size_t)l * n + k], qs[l]);
}

/*
 * Fast basis conversion from the source basis {s_i} (product D) to target primes {t_m},
 * without correction of the D-multiple:
 *   y_i = [x_i * (D/s_i)^{-1}]_{s_i}  in [0, s_i),
 *   out_m = ( sum_i y_i * (D/s_i) ) mod t_m.
 * in: [n_src][n], out: [n_dst][n].
 */
void orc_fast_base_conv(const uint64_t *in, size_t n, const uint64_t *src, int n_src,
                        const uint64_t *dst, int n_dst, uint64_t *out) {
    uint64_t *dhat_inv = (uint64_t *)malloc(sizeof(uint64_t) * n_src);
    uint64_t *dhat_mod = (uint64_t *)malloc(sizeof(uint64_t) * n_src * n_dst);
    for (int i = 0; i < n_src; i++) {
        uint64_t h = 1; /* (D / s_i) mod s_i */
        for (int j = 0; j < n_src; j++) if (j != i) h = mulmod(h, src[j] % src[i], src[i]);
        dhat_inv[i] = invmod(h, src[i]);
        for (int m = 0; m < n_dst; m++) {
            uint64_t hm = 1 % dst[m]; /* (D / s_i) mod t_m */
            for (int j = 0; j < n_src; j++) if (j != i) hm = mulmod(hm, src[j] % dst[m], dst[m]);
            dhat_mod[i * n_dst + m] = hm;
        }
    }
#pragma omp parallel for
    for (int m = 0; m < n_dst; m++) {
        uint64_t tm = dst[m];
        for (size_t k = 0; k < n; k++) {
            uint64_t acc = 0;
            for (int i = 0; i < n_src; i++) {
                uint64_t y = mulmod(in[(size_t)i * n + k], dhat_inv[i], src[i]);
                acc = addmod(acc, mulmod(y % tm, dhat_mod[i * n_dst + m], tm), tm);
            }
            out[(size_t)m * n + k] = acc;
        }
    }
    free(dhat_inv);
    free(dhat_mod);
}

/*
 * The same conversion with centred terms: y_i is replaced by y_i - s_i when
 * y_i > (s_i - 1)/2, so the sum sum_i y_i (D/s_i) lies in (-n_src D/2, n_src D/2] and
 * differs from the centred representative of x mod D by a multiple u D with u of
 * mean zero:
 *   out_m = ( sum_i y_i (D/s_i) - #{i : y_i > (s_i-1)/2} * D ) mod t_m.
 */
void orc_fast_base_conv_centered(const uint64_t *in, size_t n, const uint64_t *src, int n_src,
                                 const uint64_t *dst, int n_dst, uint64_t *out) {
    orc_fast_base_conv(in, n, src, n_src, dst, n_dst, out);
    uint64_t *dhat_inv = (uint64_t *)malloc(sizeof(uint64_t) * n_src);
    for (int i = 0; i < n_src; i++) {
        uint64_t h = 1;
        for (int j = 0; j < n_src; j++) if (j != i) h = mulmod(h, src[j] % src[i], src[i]);
        dhat_inv[i] = invmod(h, src[i]);
    }
#pragma omp parallel for
    for (int m = 0; m < n_dst; m++) {
        uint64_t tm = dst[m];
        uint64_t Dm = 1 % tm; /* D mod t_m */
        for (int j = 0; j < n_src; j++) Dm = mulmod(Dm, src[j] % tm, tm);
        for (size_t k = 0; k < n; k++) {
            uint64_t acc = out[(size_t)m * n + k];
            for (int i = 0; i < n_src; i++) {
                uint64_t y = mulmod(in[(size_t)i * n + k], dhat_inv[i], src[i]);
                if (y > (src[i] - 1) / 2) acc = submod(acc, Dm, tm);
            }
            out[(size_t)m * n + k] = acc;
        }
    }
    free(dhat_inv);
}

/* Seeded uniform half of a switching key.  SplitMix64 (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", 2014), from its published
 * definition: the state advances by the odd constant GAMMA and each output is the
 * state passed through the generator's mixing function, so element c of the
 * stream from seed s is mix(s + (c + 1) GAMMA).  Word (p, i) of digit j -- prime
 * index p in q_0..q_L, p_0..p_{alpha-1} (T of them), evaluation index i -- is
 * element (j T + p) n + i, taken into [0, q_p) as the high word of x q_p.  The
 * value is the Montgomery form a 2^64 mod q_p of the key's a at that evaluation. */
static uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void orc_seeded_key_a(uint64_t seed, int j, int T, const uint64_t *primes, int np, size_t n, uint64_t *out) {
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
#pragma omp parallel for
    for (int p = 0; p < np; p++) {
        for (size_t i = 0; i < n; i++) {
            const uint64_t c = ((uint64_t)j * (uint64_t)T + (uint64_t)p) * (uint64_t)n + i;
            const uint64_t x = sm64_mix(seed + (c + 1) * gamma);
            out[(size_t)p * n + i] = (uint64_t)(((u128)x * primes[p]) >> 64);
        }
    }
}

/* Basis conversion with the multiple of D decided by one rounding: for source
 * residues x_i (basis s_i, D = prod s_i), y_i = x_i (D/s_i)^-1 mod s_i in [0, s_i),
 * f = sum_i y_i * (1/s_i) in IEEE double (each product and sum rounded to nearest,
 * in source order, 1/s_i the correctly rounded reciprocal), v = floor(f + 1/2), and
 *   out_m = ( sum_i y_i (D/s_i) - v D ) mod t_m,
 * the centred representative of x mod D (the exact one unless f lies within double
 * rounding of a half-integer). */
void orc_base_conv_rounded(const uint64_t *in, size_t n, const uint64_t *src, int n_src,
                           const uint64_t *dst, int n_dst, uint64_t *out) {
    uint64_t *dhat_inv = (uint64_t *)malloc(sizeof(uint64_t) * n_src);
    double *rcp = (double *)malloc(sizeof(double) * n_src);
    for (int i = 0; i < n_src; i++) {
        uint64_t h = 1;
        for (int j = 0; j < n_src; j++) if (j != i) h = mulmod(h, src[j] % src[i], src[i]);
        dhat_inv[i] = invmod(h, src[i]);
        rcp[i] = 1.0 / (double)src[i];
    }
    int64_t *v = (int64_t *)malloc(sizeof(int64_t) * n);
#pragma omp parallel for
    for (size_t k = 0; k < n; k++) {
        double f = 0.0;
        for (int i = 0; i < n_src; i++) {
            const uint64_t y = mulmod(in[(size_t)i * n + k], dhat_inv[i], src[i]);
            const double p = (double)y * rcp[i];
            f = f + p;
        }
        v[k] = (int64_t)floor(f + 0.5);
    }
#pragma omp parallel for
    for (int m = 0; m < n_dst; m++) {
        uint64_t tm = dst[m];
        uint64_t Dm = 1 % tm;
        for (int j = 0; j < n_src; j++) Dm = mulmod(Dm, src[j] % tm, tm);
        for (size_t k = 0; k < n; k++) {
            uint64_t acc = 0;
            for (int i = 0; i < n_src; i++) {
                uint64_t dh = 1 % tm;   /* D / s_i mod t_m */
                for (int j = 0; j < n_src; j++) if (j != i) dh = mulmod(dh, src[j] % tm, tm);
                const uint64_t y = mulmod(in[(size_t)i * n + k], dhat_inv[i], src[i]);
                acc = addmod(acc, mulmod(y % tm, dh, tm), tm);
            }
            acc = submod(acc, mulmod((uint64_t)v[k] % tm, Dm, tm), tm);
            out[(size_t)m * n + k] = acc;
        }
    }
    free(v);
    free(rcp);
    free(dhat_inv);
}
