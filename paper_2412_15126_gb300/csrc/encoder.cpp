// Canonical-embedding encoder and decoder on the host (Sec. 2.1: a plaintext
// polynomial carries n/2 complex slots).  Slot j is the evaluation at
// zeta^(5^j), zeta = exp(i pi / n).  The transform is a radix-2 complex FFT.
#include <cmath>
#include <complex>
#include <vector>

#include "rk_internal.cuh"

namespace {
typedef std::complex<double> cd;

// In-place radix-2 FFT: sign = -1 computes sum_t x_t e^{-2 pi i t k / n}, +1 the conjugate kernel.
void fft(std::vector<cd>& a, int sign) {
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; i++) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    std::vector<cd> root(n / 2);
    for (size_t k = 0; k < n / 2; k++) {
        double ang = sign * 2.0 * M_PI * (double)k / (double)n;
        root[k] = cd(std::cos(ang), std::sin(ang));
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const size_t step = n / len;
        for (size_t i = 0; i < n; i += len) {
            for (size_t k = 0; k < len / 2; k++) {
                cd u = a[i + k], v = a[i + k + len / 2] * root[k * step];
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
        }
    }
}
}  // namespace

void encode_unscaled(int log_n, const double* z, size_t count, std::vector<double>& u) {
    const size_t n = (size_t)1 << log_n, slots = n / 2, two_n = 2 * n;
    std::vector<cd> vals(n, cd(0, 0));   // vals[t] = u(zeta^(2t+1))
    size_t e = 1;
    for (size_t j = 0; j < slots; j++) {
        const double zj = j < count ? z[j] : 0.0;
        vals[(e - 1) / 2] = cd(zj, 0);
        vals[(two_n - e - 1) / 2] = cd(zj, 0);   // conjugate point, real slot values
        e = (e * 5) % two_n;
    }
    fft(vals, -1);                               // a_k = u_k zeta^k  (times n)
    u.resize(n);
    for (size_t k = 0; k < n; k++) {
        double ang = -M_PI * (double)k / (double)n;
        cd a = vals[k] / (double)n;
        u[k] = (a * cd(std::cos(ang), std::sin(ang))).real();
    }
}

void decode_coeffs(int log_n, const std::vector<double>& m, std::vector<double>& slots_out) {
    const size_t n = (size_t)1 << log_n, slots = n / 2, two_n = 2 * n;
    std::vector<cd> a(n);
    for (size_t k = 0; k < n; k++) {
        double ang = M_PI * (double)k / (double)n;
        a[k] = m[k] * cd(std::cos(ang), std::sin(ang));
    }
    fft(a, +1);                                  // vals[t] = m(zeta^(2t+1))
    slots_out.resize(slots);
    size_t e = 1;
    for (size_t j = 0; j < slots; j++) {
        slots_out[j] = a[(e - 1) / 2].real();
        e = (e * 5) % two_n;
    }
}
