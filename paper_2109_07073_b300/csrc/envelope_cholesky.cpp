// In-place L L^T factorisation of the symmetric positive definite pose system,
// stored by its lower envelope (skyline) in 6 x 6 pose blocks: row r holds
// columns first[r] .. r at a[off[r] + (c - first[r])], and the six rows of a
// pose share their first column (a multiple of 6).
//
// Block-row order: for block row I and each block column J of its envelope,
// the 36 dot products of I's rows with J's rows over their common columns
// before J form one small product, computed with independent accumulators
// (four doubles at a time on hosts with AVX2 and FMA, chosen at run time;
// VGICP_HOST_SIMD=0 in the environment selects the portable loops);
// the few terms inside block J follow column by column (the six rows of a
// column are independent), each scaled by its pivot's reciprocal.  Entry by entry, the same sums as the textbook row algorithm, in a
// different order; the dependent chain of the row algorithm (each entry's
// dot product waits for the entry before it) is what the blocking removes.
#include "envelope_cholesky.h"

#include <immintrin.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>

namespace vg {

namespace {

// C[r][c] = sum over k < len of x_r[k] y_c[k], x_r = xs[r], y_c = ys[c] (6 each).
inline void gram6_plain(const double *const xs[6], const double *const ys[6], int64_t len, double C[6][6])
{
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) {
            const double *x = xs[r], *y = ys[c];
            double s0 = 0.0, s1 = 0.0;
            int64_t k = 0;
            for (; k + 2 <= len; k += 2) {
                s0 += x[k] * y[k];
                s1 += x[k + 1] * y[k + 1];
            }
            if (k < len) s0 += x[k] * y[k];
            C[r][c] = s0 + s1;
        }
}

__attribute__((target("avx2,fma"))) inline double hsum(__m256d v)
{
    const __m128d h = _mm_add_pd(_mm256_castpd256_pd128(v), _mm256_extractf128_pd(v, 1));
    return _mm_cvtsd_f64(h) + _mm_cvtsd_f64(_mm_unpackhi_pd(h, h));
}

__attribute__((target("avx2,fma"))) inline void gram6_avx2(const double *const xs[6], const double *const ys[6],
                                                           int64_t len, double C[6][6])
{
    const int64_t l4 = len & ~(int64_t)3;
    for (int r = 0; r < 6; ++r) {
        const double *x = xs[r];
        __m256d acc[6];
        for (int c = 0; c < 6; ++c) acc[c] = _mm256_setzero_pd();
        for (int64_t k = 0; k < l4; k += 4) {
            const __m256d xv = _mm256_loadu_pd(x + k);
            for (int c = 0; c < 6; ++c) acc[c] = _mm256_fmadd_pd(xv, _mm256_loadu_pd(ys[c] + k), acc[c]);
        }
        for (int c = 0; c < 6; ++c) {
            double s = hsum(acc[c]);
            for (int64_t k = l4; k < len; ++k) s += x[k] * ys[c][k];
            C[r][c] = s;
        }
    }
}

template <void (*GRAM)(const double *const *, const double *const *, int64_t, double (*)[6])>
__attribute__((always_inline)) inline bool factor_blocks(double *a, const int64_t *first, const int64_t *off,
                                                         int64_t n)
{
    const int64_t nb = n / 6;
    for (int64_t I = 0; I < nb; ++I) {
        const int64_t fI = first[6 * I];
        double *ri[6];                                    // row 6I + r, indexed by column
        for (int r = 0; r < 6; ++r) ri[r] = a + off[6 * I + r] - fI;
        for (int64_t J = fI / 6; J <= I; ++J) {
            const int64_t fJ = first[6 * J], k0 = std::max(fI, fJ), k1 = 6 * J;
            const double *rj[6];
            for (int c = 0; c < 6; ++c) rj[c] = a + off[6 * J + c] - fJ;
            double C[6][6];
            const double *xs[6], *ys[6];
            for (int q = 0; q < 6; ++q) {
                xs[q] = ri[q] + k0;
                ys[q] = rj[q] + k0;
            }
            GRAM(xs, ys, k1 - k0, C);
            // the entries in block J, column by column: the six rows of a column are
            // independent of each other (each needs its own row's earlier columns)
            for (int c = 0; c < 6; ++c) {
                const int64_t j = 6 * J + c;
                int r0 = 0;
                if (J == I) {                             // the diagonal entry first: it is the pivot below
                    double s = ri[c][j] - C[c][c];
                    for (int64_t k = k1; k < j; ++k) s -= ri[c][k] * ri[c][k];
                    if (!(s > 0.0)) return false;
                    ri[c][j] = std::sqrt(s);
                    r0 = c + 1;
                }
                const double inv = 1.0 / rj[c][j];
                for (int r = r0; r < 6; ++r) {
                    double s = ri[r][j] - C[r][c];
                    for (int64_t k = k1; k < j; ++k) s -= ri[r][k] * rj[c][k];
                    ri[r][j] = s * inv;
                }
            }
        }
    }
    return true;
}

__attribute__((target("avx2,fma"))) bool factor_avx2(double *a, const int64_t *first, const int64_t *off, int64_t n)
{
    return factor_blocks<gram6_avx2>(a, first, off, n);
}

bool factor_plain(double *a, const int64_t *first, const int64_t *off, int64_t n)
{
    return factor_blocks<gram6_plain>(a, first, off, n);
}

// AVX2 and FMA present, and not switched off with VGICP_HOST_SIMD=0 in the
// environment (read once).
bool host_has_avx2_fma()
{
    const char *env = std::getenv("VGICP_HOST_SIMD");
    if (env && env[0] == '0') return false;
    __builtin_cpu_init();
    return __builtin_cpu_supports("avx2") && __builtin_cpu_supports("fma");
}

}  // namespace

bool envelope_cholesky6(double *a, const int64_t *first, const int64_t *off, int64_t n)
{
    if (n % 6) return false;
    for (int64_t r = 0; r < n; ++r)
        if (first[r] != first[r - r % 6] || first[r] % 6 || first[r] > r - r % 6) return false;
    static const bool simd = host_has_avx2_fma();
    return simd ? factor_avx2(a, first, off, n) : factor_plain(a, first, off, n);
}

}  // namespace vg
