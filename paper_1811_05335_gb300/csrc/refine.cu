// The direct fp64 sum f_j = sum_{k=-M/2}^{M/2-1} fhat_k e^{2 pi i k x_j} (eq:nfft) and the
// residual-correction sweep of an inverse-NFFT estimate built on it,
//   fhat <- fhat + D^* F^* B_opt^* (f - A fhat)
// (the modified adjoint NFFT of eq:approx_ansatz2 as an approximate inverse of A in a
// Richardson iteration for A fhat = f, eq:problem_infft).
//
// One thread per node: the exponentials e^{2 pi i k x_j} advance by one complex rotation per
// frequency and restart from an exactly reduced sincospi every NDFT_RUN frequencies (2 k x_j is
// split by an FMA into hi + lo, hi is reduced modulo 2 exactly, lo enters to first order);
// the coefficients are staged in shared memory and read as broadcasts.  O(N M) fp64 work,
// bound by the fp64 pipe.
#include "plan.h"

namespace {

constexpr int NDFT_THREADS = 256;
constexpr int NDFT_CHUNK = 1024;   // coefficients staged per pass
constexpr int NDFT_RUN = 32;       // frequencies between exact restarts

constexpr double PI_R = 3.141592653589793;

// (cos, sin)(2 pi k x) with 2 k x = hi + lo exactly and hi reduced modulo 2 exactly
INFFT_D void exp2pi(int k, double x, double& c, double& s) {
    const double K = 2.0 * (double)k;
    const double hi = K * x;
    const double lo = fma(K, x, -hi);
    const double hr = hi - 2.0 * rint(0.5 * hi);
    double sn, cs;
    sincospi(hr, &sn, &cs);
    const double e = PI_R * lo;
    s = fma(e, cs, sn);
    c = fma(-e, sn, cs);
}

// out_j = A fhat (resid == nullptr) or resid_j - (A fhat)_j
__global__ void __launch_bounds__(NDFT_THREADS) k_ndft(const double* __restrict__ x, const double2* __restrict__ fhat,
                                                       int N, int M, const double2* __restrict__ resid,
                                                       double2* __restrict__ out) {
    __shared__ double2 cs[NDFT_CHUNK];
    const int j = blockIdx.x * NDFT_THREADS + threadIdx.x;
    const double xj = j < N ? x[j] : 0.0;
    double wc, ws;
    exp2pi(1, xj, wc, ws);                          // one frequency step
    double ar = 0.0, ai = 0.0;
    for (int c0 = 0; c0 < M; c0 += NDFT_CHUNK) {
        const int cn = min(NDFT_CHUNK, M - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < cn; t += NDFT_THREADS) cs[t] = fhat[c0 + t];
        __syncthreads();
        for (int b = 0; b < cn; b += NDFT_RUN) {
            double zr, zi;
            exp2pi(c0 + b - M / 2, xj, zr, zi);
            const int e = min(NDFT_RUN, cn - b);
            for (int u = 0; u < e; ++u) {
                const double2 v = cs[b + u];
                ar = fma(v.x, zr, fma(-v.y, zi, ar));
                ai = fma(v.x, zi, fma(v.y, zr, ai));
                const double t = fma(zr, wc, -zi * ws);
                zi = fma(zr, ws, zi * wc);
                zr = t;
            }
        }
    }
    if (j < N) {
        if (resid) {
            const double2 f = resid[j];
            out[j] = make_double2(f.x - ar, f.y - ai);
        } else {
            out[j] = make_double2(ar, ai);
        }
    }
}

__global__ void k_axpy_z(double2* __restrict__ y, const double2* __restrict__ d, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double2 a = y[i], b = d[i];
        y[i] = make_double2(a.x + b.x, a.y + b.y);
    }
}

}  // namespace

cudaError_t run_ndft_z(Plan* p, const void* fhat, const void* resid, void* out, cudaStream_t s) {
    const int N = (int)p->N, M = (int)p->M;
    launch_begin(p, "ndft_z", s);
    k_ndft<<<(N + NDFT_THREADS - 1) / NDFT_THREADS, NDFT_THREADS, 0, s>>>(p->x, (const double2*)fhat, N, M,
                                                                          (const double2*)resid, (double2*)out);
    launch_end(p, s);
    return cudaGetLastError();
}

cudaError_t run_axpy_z(Plan* p, void* y, const void* d, int n, cudaStream_t s) {
    launch_begin(p, "axpy_z", s);
    k_axpy_z<<<(n + 255) / 256, 256, 0, s>>>((double2*)y, (const double2*)d, n);
    launch_end(p, s);
    return cudaGetLastError();
}

// ---- the NFFT of Sec. 2.1 with a Kaiser-Bessel window --------------------------------
//
// f_j ~ sum_l g_l w~(x_j - l/M_sigma), g = F D fhat, D = diag(1/(M_sigma w^(k))), the window
// truncated to |x| <= KB_M/M_sigma.  Window (Kaiser-Bessel, as used throughout the NFFT
// literature): with t = M_sigma x and b = pi (2 - 1/sigma),
//   w(x) = sinh(b sqrt(KB_M^2 - t^2)) / (pi sqrt(KB_M^2 - t^2)),
//   M_sigma w^(k) = I_0(KB_M sqrt(b^2 - (2 pi k/M_sigma)^2)),
// I_0 by its power series (all terms positive).  With sigma = 2 and KB_M = 12 the truncation
// error, of order exp(-2 pi KB_M sqrt(1 - 1/sigma)), is far below fp64 rounding.

namespace {

constexpr int KB_M = 12;

INFFT_D double bessel_i0(double z) {
    const double q = 0.25 * z * z;
    double term = 1.0, sum = 1.0;
    for (int j = 1; j < 200; ++j) {
        term *= q / ((double)j * (double)j);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

// coef[k + M/2] = fhat[k + M/2] / (M_sigma w^(k))
__global__ void k_kb_deconv(const double2* __restrict__ fhat, int M, int Ms, double b, double2* __restrict__ coef) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const double a = 2.0 * PI_R * (double)(i - M / 2) / (double)Ms;
    const double d = 1.0 / bessel_i0((double)KB_M * sqrt(b * b - a * a));
    const double2 v = fhat[i];
    coef[i] = make_double2(v.x * d, v.y * d);
}

// out_j = sum_l g_{l + Ms/2} w(x_j - l/Ms) (or resid_j minus it), one thread per node
__global__ void k_kb_gather(const double* __restrict__ x, const double2* __restrict__ g, int N, int Ms, double b,
                            const double2* __restrict__ resid, double2* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double u = (double)Ms * x[j];              // exact: Ms is a power of two
    const int lo = (int)ceil(u) - KB_M, hi = (int)floor(u) + KB_M;
    const double mm = (double)(KB_M * KB_M);
    double ar = 0.0, ai = 0.0;
    for (int l = lo; l <= hi; ++l) {
        const double t = u - (double)l;              // exact
        const double s = sqrt(fmax(mm - t * t, 0.0));
        const double bs = b * s;
        const double w = (bs < 1e-6 ? b * fma(bs * bs, 1.0 / 6.0, 1.0) : sinh(bs) / s) * (1.0 / PI_R);
        int p = (l + Ms / 2) % Ms;
        if (p < 0) p += Ms;
        const double2 v = g[p];
        ar = fma(w, v.x, ar);
        ai = fma(w, v.y, ai);
    }
    if (resid) {
        const double2 f = resid[j];
        out[j] = make_double2(f.x - ar, f.y - ai);
    } else {
        out[j] = make_double2(ar, ai);
    }
}

}  // namespace

bool nfft_kb_supported(const Plan* p) { return p->Ms >= 2 * p->M && p->Ms >= 8 * KB_M && !(p->Ms & (p->Ms - 1)); }

cudaError_t run_nfft_kb_z(Plan* p, const void* fhat, const void* resid, void* out, void* coef, cudaStream_t s) {
    const int N = (int)p->N, M = (int)p->M, Ms = (int)p->Ms;
    const double b = PI_R * (2.0 - (double)M / (double)Ms);   // pi (2 - 1/sigma)
    launch_begin(p, "kb_deconv_z", s);
    k_kb_deconv<<<(M + 255) / 256, 256, 0, s>>>((const double2*)fhat, M, Ms, b, (double2*)coef);
    launch_end(p, s);
    cudaError_t e = run_fft_forward_band_z(p, coef, p->grid, s);
    if (e != cudaSuccess) return e;
    launch_begin(p, "kb_gather_z", s);
    k_kb_gather<<<(N + 255) / 256, 256, 0, s>>>(p->x, (const double2*)p->grid, N, Ms, b, (const double2*)resid,
                                                (double2*)out);
    launch_end(p, s);
    return cudaGetLastError();
}
