/* CPU apply of the modified adjoint NFFT, fhat = D^* F^* B_opt^* f (Sec. 3.2.2,
 * eq:approx_ansatz2), in plain C with OpenMP: test infrastructure of the oracle (a second,
 * independent evaluation of the oracle's numpy apply) and the multi-core CPU baseline
 * the benchmark times.  It shares nothing with the CUDA library.
 *
 *   g_l   = sum_{j in I(l)} b_{l,j} f_j          gather per grid point, B_opt in the oracle's
 *                                                CSR layout (ptr[l] .. ptr[l+1] over idx, b)
 *   h_k   = sum_l g_l exp(-2 pi i k l / M_sigma) one length-M_sigma radix-2 FFT over the grid
 *                                                index p = l + M_sigma/2, then
 *                                                h_k = (-1)^k DFT(g)[k mod M_sigma]
 *   fhat_k = d_k h_k                             d_k = 1/M_sigma (kernel full), 0 at
 *                                                k = -M/2 for kernel sym (eq:matrix_D)
 *
 * The FFT is the iterative decimation-in-time radix-2 Cooley-Tukey algorithm (bit-reversal
 * permutation, then log2(M_sigma) butterfly stages), twiddles from a table of
 * exp(-2 pi i t / M_sigma), t < M_sigma/2, evaluated with cos/sin of the exact fraction.
 * M_sigma must be a power of two.  Complex arrays are interleaved (re, im). */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int capply_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the following calls (n >= 1) */
void capply_set_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static int64_t bit_reverse(int64_t v, int bits) {
    int64_t r = 0;
    for (int i = 0; i < bits; ++i) {
        r = (r << 1) | (v & 1);
        v >>= 1;
    }
    return r;
}

/* tw[2t], tw[2t+1] = cos, sin of -2 pi t / Ms for t < Ms/2 */
void capply_twiddles(int64_t Ms, double* tw) {
    const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < Ms / 2; ++t) {
        const double a = -two_pi * ((double)t / (double)Ms);
        tw[2 * t] = cos(a);
        tw[2 * t + 1] = sin(a);
    }
}

#define DEFINE_APPLY(NAME, REAL)                                                                        \
    int NAME(int64_t Ms, int64_t M, int sym, const int64_t* ptr, const int64_t* idx, const double* b,   \
             const REAL* f, REAL* fhat, REAL* work, const double* tw) {                                 \
        int bits = 0;                                                                                   \
        while (((int64_t)1 << bits) < Ms) ++bits;                                                       \
        if (((int64_t)1 << bits) != Ms || M > Ms || (M & 1)) return 1;                                  \
        /* spread, written straight to its bit-reversed position */                                     \
        _Pragma("omp parallel for schedule(static)")                                                    \
        for (int64_t l = 0; l < Ms; ++l) {                                                              \
            REAL re = 0, im = 0;                                                                        \
            for (int64_t e = ptr[l]; e < ptr[l + 1]; ++e) {                                             \
                const REAL w = (REAL)b[e];                                                              \
                re += w * f[2 * idx[e]];                                                                \
                im += w * f[2 * idx[e] + 1];                                                            \
            }                                                                                           \
            const int64_t q = bit_reverse(l, bits);                                                     \
            work[2 * q] = re;                                                                           \
            work[2 * q + 1] = im;                                                                       \
        }                                                                                               \
        /* butterflies of span h = 1, 2, 4, ...: the twiddle of position j in a span is tw[j Ms/2h] */ \
        for (int64_t h = 1; h < Ms; h <<= 1) {                                                          \
            const int64_t stride = Ms / (2 * h);                                                        \
            _Pragma("omp parallel for schedule(static)")                                                \
            for (int64_t t = 0; t < Ms / 2; ++t) {                                                      \
                const int64_t blk = t / h, j = t - blk * h;                                             \
                const int64_t i0 = blk * 2 * h + j, i1 = i0 + h;                                        \
                const REAL wr = (REAL)tw[2 * j * stride], wi = (REAL)tw[2 * j * stride + 1];            \
                const REAL xr = work[2 * i1] * wr - work[2 * i1 + 1] * wi;                              \
                const REAL xi = work[2 * i1] * wi + work[2 * i1 + 1] * wr;                              \
                const REAL ar = work[2 * i0], ai = work[2 * i0 + 1];                                    \
                work[2 * i0] = ar + xr;                                                                 \
                work[2 * i0 + 1] = ai + xi;                                                             \
                work[2 * i1] = ar - xr;                                                                 \
                work[2 * i1 + 1] = ai - xi;                                                             \
            }                                                                                           \
        }                                                                                               \
        const REAL inv = (REAL)(1.0 / (double)Ms);                                                      \
        _Pragma("omp parallel for schedule(static)")                                                    \
        for (int64_t kk = 0; kk < M; ++kk) {                                                            \
            const int64_t k = kk - M / 2;                                                               \
            const int64_t q = ((k % Ms) + Ms) % Ms;                                                     \
            REAL d = (k & 1) ? -inv : inv;                                                              \
            if (sym && k == -M / 2) d = 0;                                                              \
            fhat[2 * kk] = d * work[2 * q];                                                             \
            fhat[2 * kk + 1] = d * work[2 * q + 1];                                                     \
        }                                                                                               \
        return 0;                                                                                       \
    }

DEFINE_APPLY(capply_f64, double)
DEFINE_APPLY(capply_f32, float)
