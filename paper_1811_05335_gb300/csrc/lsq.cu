// Precomputation of B_opt (Sec. 3.2.2, eq:opt_ansatz2 .. eq:solution_ansatz2).
//
// For every grid point l the real coefficients b_l on I(l) minimise
// ||L_l b - e_l||^2 + mu ||b||^2, L_l = F D H_l (eq:matrix_Ll) with the Dirichlet
// choice (Remark remark:Dirichlet_ansatz2).  Because F^* F = M_sigma I_M, the
// normal matrix has the closed form Re G_{jj'} = Re kappa(x_j - x_j') and the
// right-hand side Re r_j = Re kappa(l/M_sigma - x_j), where
//   full: Re kappa(t) = cos(pi t) sin(pi M t) / (M_sigma sin(pi t)),
//   sym : Re kappa(t) = sin(pi (M-1) t) / (M_sigma sin(pi t))   (eq:kernel_Dirichlet).
// mu = tau * Re kappa(0) (Tikhonov; the paper assumes full rank).  The systems
// are solved in fp64 by Cholesky; a failed pivot retries with mu * 1e3 (twice)
// and is counted as a fallback column.
//
// Columns with |I(l)| <= 32 are solved by one warp each (lanes own rows);
// larger columns go to a device-side list consumed by a CTA-per-column kernel.
#include "plan.h"

namespace {

struct KernelParams {
    double M;        // number of frequencies (as a double)
    double inv_Ms;   // 1 / M_sigma
    double diag;     // Re kappa(0)
    int sym;         // 0: full, 1: sym
};

// Re kappa(a - b) with a - b taken on the torus R/Z (both kernels are 1-periodic).
// Shifting each operand by 1/2 before subtracting keeps the difference of two
// points that are close across the seam x = +-1/2 exact; subtracting first and
// wrapping afterwards would lose ~11 digits and can make Re G_l + mu I indefinite.
INFFT_D double re_kappa(double a, double b, const KernelParams& kp) {
    double t = a - b;
    if (t > 0.5) t = (a - 0.5) - (b + 0.5);
    else if (t < -0.5) t = (a + 0.5) - (b - 0.5);
    if (t == 0.0) return kp.diag;
    double s, c;
    sincospi(t, &s, &c);
    if (kp.sym) return sinpi((kp.M - 1.0) * t) / s * kp.inv_Ms;
    return c * sinpi(kp.M * t) / s * kp.inv_Ms;
}

// (i, j), j <= i, of the e-th entry of a row-major lower triangle
INFFT_D void tri_index(int e, int& i, int& j) {
    int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    while (r * (r + 1) / 2 > e) --r;
    i = r;
    j = e - r * (r + 1) / 2;
}

// One warp per column; lane t owns rows t, t + 32, ... (NMAX / 32 rows).  The
// column comes from `list` (a device work list) or, when list == nullptr, is the
// warp's global index.  Columns too large for this tier are pushed to `next_list`
// (count at counters[next_counter]).
template <int NMAX, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_lsq_warp(const double* __restrict__ xs, const int32_t* __restrict__ col_start,
           const int32_t* __restrict__ col_count, const int32_t* __restrict__ col_off, int N, int Ms,
           KernelParams kp, double mu0, double* __restrict__ w64, float* __restrict__ w32,
           double* __restrict__ Jout, uint8_t* __restrict__ wide, const int32_t* __restrict__ list,
           int list_counter,
           int32_t* __restrict__ next_list, int next_counter, int32_t* __restrict__ counters) {
    constexpr int ROWS = NMAX / 32;
    constexpr int LD = NMAX + 1;     // padded row stride: conflict-free column access
    extern __shared__ double lsq_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* A = lsq_smem + (size_t)wid * (NMAX * LD + 2 * NMAX);
    double* r = A + NMAX * LD;
    double* xl = r + NMAX;
    const int total = list ? counters[list_counter] : Ms;
    for (int it = blockIdx.x * WARPS + wid; it < total; it += gridDim.x * WARPS) {
        const int p = list ? list[it] : it;
        const int n = col_count[p];
        if (n == 0) {
            if (lane == 0) { Jout[p] = 1.0; wide[p] = 0; }
            continue;
        }
        if (n > NMAX) {
            if (lane == 0) next_list[atomicAdd(&counters[next_counter], 1)] = p;
            continue;
        }
        const int s = col_start[p], off = col_off[p];
        const double tl = (double)(p - Ms / 2) / (double)Ms;   // l / M_sigma
        for (int i = lane; i < n; i += 32) {
            int q = s + i;
            if (q >= N) q -= N;
            xl[i] = xs[q];
        }
        __syncwarp();
        const int ntri = n * (n + 1) / 2;
        double mu = mu0;
        bool ok = false;
        for (int attempt = 0; attempt < 3 && !ok; ++attempt) {
            for (int i = lane; i < n; i += 32) r[i] = re_kappa(tl, xl[i], kp);
            for (int e = lane; e < ntri; e += 32) {
                int i, j;
                tri_index(e, i, j);
                A[i * LD + j] = (i == j) ? kp.diag + mu : re_kappa(xl[i], xl[j], kp);
            }
            __syncwarp();
            ok = true;
            for (int k = 0; k < n; ++k) {
                const double akk = A[k * LD + k];
                if (!(akk > 0.0) || !isfinite(akk)) { ok = false; break; }   // warp-uniform
                const double dk = sqrt(akk);
                double lik[ROWS];
#pragma unroll
                for (int t = 0; t < ROWS; ++t) {
                    const int i = lane + 32 * t;
                    lik[t] = (i > k && i < n) ? A[i * LD + k] / dk : 0.0;
                }
                __syncwarp();
#pragma unroll
                for (int t = 0; t < ROWS; ++t) {
                    const int i = lane + 32 * t;
                    if (i > k && i < n) A[i * LD + k] = lik[t];
                }
                if (lane == (k & 31)) A[k * LD + k] = dk;
                __syncwarp();
#pragma unroll
                for (int t = 0; t < ROWS; ++t) {
                    const int i = lane + 32 * t;
                    if (i > k && i < n)
                        for (int j = k + 1; j <= i; ++j) A[i * LD + j] -= lik[t] * A[j * LD + k];
                }
                __syncwarp();
            }
            if (!ok) mu *= 1e3;
        }
        if (!ok) {   // give up: empty contribution, counted as a fallback
            for (int i = lane; i < n; i += 32) { w64[off + i] = 0.0; w32[off + i] = 0.0f; }
            if (lane == 0) { Jout[p] = 1.0; wide[p] = 0; atomicAdd(&counters[CNT_FALLBACK], 1); }
            continue;
        }
        if (lane == 0 && mu != mu0) atomicAdd(&counters[CNT_FALLBACK], 1);
        // forward: y = L^{-1} r (r overwritten by y); ||y||^2 = r . b
        double ysq = 0.0;
        for (int k = 0; k < n; ++k) {
            const double yk = r[k] / A[k * LD + k];
            ysq += yk * yk;
            __syncwarp();
            if (lane == (k & 31)) r[k] = yk;
#pragma unroll
            for (int t = 0; t < ROWS; ++t) {
                const int i = lane + 32 * t;
                if (i > k && i < n) r[i] -= A[i * LD + k] * yk;
            }
            __syncwarp();
        }
        // backward: L^T b = y (r overwritten by b)
        for (int k = n - 1; k >= 0; --k) {
            const double bk = r[k] / A[k * LD + k];
            __syncwarp();
            if (lane == (k & 31)) r[k] = bk;
#pragma unroll
            for (int t = 0; t < ROWS; ++t) {
                const int i = lane + 32 * t;
                if (i < k) r[i] -= A[k * LD + i] * bk;
            }
            __syncwarp();
        }
        double bsq = 0.0, babs = 0.0;
        for (int i = lane; i < n; i += 32) {
            const double b = r[i];
            w64[off + i] = b;
            w32[off + i] = (float)b;
            bsq += b * b;
            babs += fabs(b);
        }
        for (int o = 16; o; o >>= 1) {
            bsq += __shfl_xor_sync(0xffffffffu, bsq, o);
            babs += __shfl_xor_sync(0xffffffffu, babs, o);
        }
        // J_l = ||L b - e_l||^2 = 1 - r.b - mu ||b||^2 at the regularised optimum
        if (lane == 0) {
            Jout[p] = 1.0 - ysq - mu * bsq;
            wide[p] = babs > WIDE_COLUMN_L1;
        }
        __syncwarp();
    }
}

template <int NMAX, int WARPS> constexpr size_t warp_smem_bytes() {
    return (size_t)WARPS * (NMAX * (NMAX + 1) + 2 * NMAX) * sizeof(double);
}

constexpr int CTA_THREADS = 256;
constexpr int CN = LSQ_CTA_NMAX;
INFFT_D int trow(int i) { return i * (i + 1) / 2; }   // packed lower-triangle row start

__global__ void __launch_bounds__(CTA_THREADS)
k_lsq_cta(const double* __restrict__ xs, const int32_t* __restrict__ col_start,
          const int32_t* __restrict__ col_count, const int32_t* __restrict__ col_off, int N, int Ms,
          KernelParams kp, double mu0, double* __restrict__ w64, float* __restrict__ w32,
          double* __restrict__ Jout, uint8_t* __restrict__ wide, const int32_t* __restrict__ big_list,
          int32_t* __restrict__ counters) {
    extern __shared__ double smem[];
    double* A = smem;                 // CN (CN + 1) / 2, packed rows
    double* r = A + CN * (CN + 1) / 2; // CN
    double* xl = r + CN;              // CN
    __shared__ int s_ok;
    __shared__ double s_red[2 * (CTA_THREADS / 32)];
    const int total = counters[CNT_BIG_LIST];   // filled by the warp tiers
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int p = big_list[it];
        const int n = col_count[p], s = col_start[p], off = col_off[p];
        if (n > CN) {
            for (int i = threadIdx.x; i < n; i += CTA_THREADS) { w64[off + i] = 0.0; w32[off + i] = 0.0f; }
            if (threadIdx.x == 0) { Jout[p] = 1.0; wide[p] = 0; atomicAdd(&counters[CNT_UNSUPPORTED], 1); }
            continue;
        }
        const double tl = (double)(p - Ms / 2) / (double)Ms;
        for (int i = threadIdx.x; i < n; i += CTA_THREADS) {
            int q = s + i;
            if (q >= N) q -= N;
            xl[i] = xs[q];
        }
        __syncthreads();
        const int ntri = n * (n + 1) / 2;
        double mu = mu0;
        bool ok = false;
        for (int attempt = 0; attempt < 3 && !ok; ++attempt) {
            for (int i = threadIdx.x; i < n; i += CTA_THREADS) r[i] = re_kappa(tl, xl[i], kp);
            for (int e = threadIdx.x; e < ntri; e += CTA_THREADS) {
                int i, j;
                tri_index(e, i, j);
                A[trow(i) + j] = (i == j) ? kp.diag + mu : re_kappa(xl[i], xl[j], kp);
            }
            if (threadIdx.x == 0) s_ok = 1;
            __syncthreads();
            for (int k = 0; k < n; ++k) {
                double akk = A[trow(k) + k];
                if (!(akk > 0.0) || !isfinite(akk)) {   // block-uniform
                    if (threadIdx.x == 0) s_ok = 0;
                    break;
                }
                double dk = sqrt(akk);
                __syncthreads();
                for (int i = k + 1 + threadIdx.x; i < n; i += CTA_THREADS) A[trow(i) + k] /= dk;
                if (threadIdx.x == 0) A[trow(k) + k] = dk;
                __syncthreads();
                const int m2 = n - k - 1;
                const int nt = m2 * (m2 + 1) / 2;
                for (int e = threadIdx.x; e < nt; e += CTA_THREADS) {
                    int a, b;
                    tri_index(e, a, b);
                    int i = k + 1 + a, j = k + 1 + b;
                    A[trow(i) + j] -= A[trow(i) + k] * A[trow(j) + k];
                }
                __syncthreads();
            }
            __syncthreads();
            ok = s_ok != 0;
            if (!ok) mu *= 1e3;
            __syncthreads();
        }
        if (!ok) {
            for (int i = threadIdx.x; i < n; i += CTA_THREADS) { w64[off + i] = 0.0; w32[off + i] = 0.0f; }
            if (threadIdx.x == 0) { Jout[p] = 1.0; wide[p] = 0; atomicAdd(&counters[CNT_FALLBACK], 1); }
            __syncthreads();
            continue;
        }
        if (threadIdx.x == 0 && mu != mu0) atomicAdd(&counters[CNT_FALLBACK], 1);
        double ysq = 0.0;
        for (int k = 0; k < n; ++k) {
            double yk = r[k] / A[trow(k) + k];
            ysq += yk * yk;
            __syncthreads();
            if (threadIdx.x == 0) r[k] = yk;
            for (int i = k + 1 + threadIdx.x; i < n; i += CTA_THREADS) r[i] -= A[trow(i) + k] * yk;
            __syncthreads();
        }
        for (int k = n - 1; k >= 0; --k) {
            double bk = r[k] / A[trow(k) + k];
            __syncthreads();
            if (threadIdx.x == 0) r[k] = bk;
            for (int i = threadIdx.x; i < k; i += CTA_THREADS) r[i] -= A[trow(k) + i] * bk;
            __syncthreads();
        }
        double bsq = 0.0, babs = 0.0;
        for (int i = threadIdx.x; i < n; i += CTA_THREADS) {
            double b = r[i];
            w64[off + i] = b;
            w32[off + i] = (float)b;
            bsq += b * b;
            babs += fabs(b);
        }
        for (int o = 16; o; o >>= 1) {
            bsq += __shfl_xor_sync(0xffffffffu, bsq, o);
            babs += __shfl_xor_sync(0xffffffffu, babs, o);
        }
        if ((threadIdx.x & 31) == 0) { s_red[threadIdx.x >> 5] = bsq; s_red[CTA_THREADS / 32 + (threadIdx.x >> 5)] = babs; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0, a = 0.0;
            for (int w = 0; w < CTA_THREADS / 32; ++w) { t += s_red[w]; a += s_red[CTA_THREADS / 32 + w]; }
            Jout[p] = 1.0 - ysq - mu * t;
            wide[p] = a > WIDE_COLUMN_L1;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t run_precompute(Plan* p, cudaStream_t s) {
    const int N = (int)p->N, Ms = (int)p->Ms;
    KernelParams kp;
    kp.M = (double)p->M;
    kp.inv_Ms = 1.0 / (double)Ms;
    kp.sym = (p->kernel == INFFT_KERNEL_SYM);
    kp.diag = (kp.sym ? (double)(p->M - 1) : (double)p->M) / (double)Ms;
    const double mu = p->tau * kp.diag;

    // clear the precompute counters (fallback, unsupported, work lists), keep the pattern's
    cudaError_t e = cudaMemsetAsync(p->counters + CNT_FALLBACK, 0, 2 * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->counters + CNT_BIG_LIST, 0, 2 * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (sms <= 0) sms = 148;

    constexpr int W1 = 4, W2 = 4;
    auto k1 = k_lsq_warp<LSQ_WARP_NMAX, W1>;
    auto k2 = k_lsq_warp<LSQ_WARP2_NMAX, W2>;
    const size_t s1 = warp_smem_bytes<LSQ_WARP_NMAX, W1>(), s2 = warp_smem_bytes<LSQ_WARP2_NMAX, W2>();
    const size_t s3 = (size_t)(CN * (CN + 1) / 2 + 2 * CN) * sizeof(double);
    if ((e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_lsq_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s3)) != cudaSuccess)
        return e;

    // tier 1: every column, |I(l)| <= 32; larger ones go to the mid list
    launch_begin(p, "lsq_warp32", s);
    k1<<<(Ms + W1 - 1) / W1, W1 * 32, s1, s>>>(p->xs, p->col_start, p->col_count, p->col_off, N, Ms, kp, mu,
                                               p->w64, p->w32, p->J, p->wide, nullptr, 0, p->mid_list, CNT_MID_LIST,
                                               p->counters);
    launch_end(p, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // tier 2: the mid list, |I(l)| <= 64; larger ones go to the big list
    launch_begin(p, "lsq_warp64", s);
    k2<<<2 * sms, W2 * 32, s2, s>>>(p->xs, p->col_start, p->col_count, p->col_off, N, Ms, kp, mu, p->w64,
                                    p->w32, p->J, p->wide, p->mid_list, CNT_MID_LIST, p->big_list, CNT_BIG_LIST,
                                    p->counters);
    launch_end(p, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // tier 3: the big list, one CTA per column, |I(l)| <= 224
    launch_begin(p, "lsq_cta", s);
    k_lsq_cta<<<sms, CTA_THREADS, s3, s>>>(p->xs, p->col_start, p->col_count, p->col_off, N, Ms, kp, mu, p->w64,
                                           p->w32, p->J, p->wide, p->big_list, p->counters);
    launch_end(p, s);
    return cudaGetLastError();
}
