// Gradient of a loss through the inverse NFFT with respect to the nodes.
//
// fhat = D^* F^* B_opt(x)^* f (eq:approx_ansatz2); w = dL/dRe fhat + i dL/dIm fhat.
// With gamma = F D w on the grid and beta_{l,i} = Re(conj(gamma_l) f_i) = dL/db_{l,i},
// implicit differentiation of every column's normal equations A_l b_l = r_l
// (A_l = Re G_l + mu I, Sec. 3.2.2, the pattern held fixed) gives, with
// lambda_l = A_l^{-1} beta_l and kappa' the derivative of Re kappa,
//   dL/dx_j = sum_{l : j in I(l)} [ -lambda_{l,j} kappa'(l/M_sigma - x_j)
//                                   - lambda_{l,j} sum_k kappa'(x_j - x_k) b_{l,k}
//                                   - b_{l,j} sum_i kappa'(x_j - x_i) lambda_{l,i} ].
// One warp per column (lanes own rows) re-factors A_l in fp64 (Gram entries as in the
// precompute), solves for lambda_l, evaluates each pair's kappa' once (it is odd) and
// writes each node's term next to the column's weights; a per-node pass sums them.
#include <cmath>
#include <cstring>

#include "lsq_device.cuh"

namespace {

struct GradParams {
    double M, inv_Ms, diag;
    int sym;
    int short_series;   // 1: every near pair has |pi t| so small that three terms of each series suffice
    double cs[10];    // kappa'(t) = t * sum_p cs[p] t^{2p} for |M t| <= 1/4 (host-folded series)
};

INFFT_D double g_torus_diff(double a, double b) {
    double t = a - b;
    if (t > 0.5) t = (a - 0.5) - (b + 0.5);
    else if (t < -0.5) t = (a + 0.5) - (b - 0.5);
    return t;
}

INFFT_D double g_recip(double u) {
    double r = (double)__frcp_rn((float)u);
    double e = fma(-u, r, 1.0);
    r = fma(r, e, r);
    e = fma(-u, r, 1.0);
    return fma(r, e, r);
}

// d/dt Re kappa(t) at t = a - b; pa, pb = (sin, cos)(pi M a), (sin, cos)(pi M b).
//   full: (pi / M_sigma) [M cot(u) cos(M u) - sin(M u) / sin^2(u)],  u = pi t
//   sym : full + (pi M / M_sigma) sin(M u)
// Branches: |M t| <= 1/4: the series of the defining sum (no cancellation);
// |t| <= 1/32: u cot u and u^2 / sin^2 u by their Taylor series (Bernoulli numbers),
// sin/cos(M u) by angle addition of the phases, a Newton reciprocal of u;
// otherwise library transcendentals.
INFFT_D double g_kappa_prime(double a, double b, double2 pa, double2 pb, const GradParams& kp) {
    const double t = g_torus_diff(a, b);
    if (t == 0.0) return 0.0;
    if (fabs(kp.M * t) <= 0.25) {
        const double t2 = t * t;
        double acc = kp.cs[9];
#pragma unroll
        for (int p = 8; p >= 0; --p) acc = fma(t2, acc, kp.cs[p]);
        double v = t * acc;
        if (kp.sym) {   // + (pi M / M_sigma) sin(pi M t), |pi M t| <= pi/4
            const double z = PI * kp.M * t, zz = z * z;
            double sz = fma(zz, 1.0 / 355687428096000.0, -1.0 / 1307674368000.0);
            sz = fma(zz, sz, 1.0 / 6227020800.0);
            sz = fma(zz, sz, -1.0 / 39916800.0);
            sz = fma(zz, sz, 1.0 / 362880.0);
            sz = fma(zz, sz, -1.0 / 5040.0);
            sz = fma(zz, sz, 1.0 / 120.0);
            sz = fma(zz, sz, -1.0 / 6.0);
            sz = fma(zz, sz, 1.0);
            v += PI * kp.M * kp.inv_Ms * z * sz;
        }
        return v;
    }
    double sinM, cosM, full;
    if (fabs(t) <= SMALL_T) {
        const double u = PI * t, w = u * u;
        double xc, q;
        if (kp.short_series) {   // uniform across the launch
            xc = fma(w, -1.0 / 45.0, -1.0 / 3.0);
            xc = fma(w, xc, 1.0);
            q = fma(w, 1.0 / 15.0, 1.0 / 3.0);
            q = fma(w, q, 1.0);
        } else {
            xc = fma(w, -4.0 / 18243225.0, -1382.0 / 638512875.0);   // u cot u
            xc = fma(w, xc, -2.0 / 93555.0);
            xc = fma(w, xc, -1.0 / 4725.0);
            xc = fma(w, xc, -2.0 / 945.0);
            xc = fma(w, xc, -1.0 / 45.0);
            xc = fma(w, xc, -1.0 / 3.0);
            xc = fma(w, xc, 1.0);
            q = fma(w, 4.0 / 1403325.0, 1382.0 / 58046625.0);         // u^2 / sin^2 u
            q = fma(w, q, 2.0 / 10395.0);
            q = fma(w, q, 1.0 / 675.0);
            q = fma(w, q, 2.0 / 189.0);
            q = fma(w, q, 1.0 / 15.0);
            q = fma(w, q, 1.0 / 3.0);
            q = fma(w, q, 1.0);
        }
        sinM = fma(pa.x, pb.y, -pa.y * pb.x);
        cosM = fma(pa.y, pb.y, pa.x * pb.x);
        const double ru = g_recip(u);
        full = PI * kp.inv_Ms * ru * (kp.M * xc * cosM - q * sinM * ru);
    } else {
        double s, c;
        sincospi(t, &s, &c);
        sincospi(kp.M * t, &sinM, &cosM);
        full = PI * kp.inv_Ms * (kp.M * (c / s) * cosM - sinM / (s * s));
    }
    if (kp.sym) full += PI * kp.M * kp.inv_Ms * sinM;
    return full;
}

constexpr int GW = 4;          // warps per CTA
constexpr int GN = 64;         // largest column handled
constexpr int GLD = GN + 1;

// Per column: rebuild A_l, Cholesky, lambda_l = A_l^{-1} beta_l, per-node terms into gterm.
__global__ void __launch_bounds__(GW * 32)
k_grad_cols(const double* __restrict__ xs, const double2* __restrict__ ph, const int32_t* __restrict__ perm,
            const int32_t* __restrict__ col_start, const int32_t* __restrict__ col_count,
            const int32_t* __restrict__ col_off, const double* __restrict__ w64, const float2* __restrict__ f,
            const float2* __restrict__ gamma, int N, int Ms, GradParams kp, KernelParams kk, double mu,
            double* __restrict__ gterm, int32_t* __restrict__ counters) {
    extern __shared__ double gsm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* A = gsm + (size_t)wid * (GN * GLD + 6 * GN);
    double* lam = A + GN * GLD;
    double* bb = lam + GN;
    double* xl = bb + GN;
    double2* pv = (double2*)(xl + GN);    // xl + GN is 16-byte aligned: GN and GLD * GN are even
    for (int p = blockIdx.x * GW + wid; p < Ms; p += gridDim.x * GW) {
        const int n = col_count[p];
        if (n == 0) continue;
        const int s = col_start[p], off = col_off[p];
        if (n > GN) {
            for (int i = lane; i < n; i += 32) gterm[off + i] = 0.0;
            if (lane == 0) atomicAdd(&counters[CNT_GRAD_FAIL], 1);
            continue;
        }
        const double tl = (double)(p - Ms / 2) / (double)Ms;
        double2 pl;
        {
            const double pp = kp.M * tl, e = fma(kp.M, tl, -pp), r = pp - 2.0 * rint(0.5 * pp);
            sincospi(r + e, &pl.x, &pl.y);
        }
        const float2 gl = gamma[p];
        for (int i = lane; i < n; i += 32) {
            int q = s + i;
            if (q >= N) q -= N;
            xl[i] = xs[q];
            pv[i] = ph[q];
            bb[i] = w64[off + i];
            const float2 fi = f[perm[q]];
            lam[i] = (double)gl.x * (double)fi.x + (double)gl.y * (double)fi.y;   // beta = Re(conj(gamma) f)
        }
        __syncwarp();
        for (int e = lane; e < n * n; e += 32) {
            const int i = e / n, j = e % n;
            if (j <= i) A[i * GLD + j] = (i == j) ? kp.diag + mu : re_kappa(xl[i], xl[j], pv[i], pv[j], kk);
        }
        __syncwarp();
        bool ok = true;
        for (int k = 0; k < n; ++k) {
            const double akk = A[k * GLD + k];
            if (!(akk > 0.0) || !isfinite(akk)) { ok = false; break; }
            const double rp = rsqrt(akk);
            double lik[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int i = lane + 32 * t;
                lik[t] = (i > k && i < n) ? A[i * GLD + k] * rp : 0.0;
            }
            __syncwarp();
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int i = lane + 32 * t;
                if (i > k && i < n) A[i * GLD + k] = lik[t];
            }
            if (lane == (k & 31)) A[k * GLD + k] = rp;
            __syncwarp();
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int i = lane + 32 * t;
                if (i > k && i < n)
                    for (int j = k + 1; j <= i; ++j) A[i * GLD + j] = fma(-lik[t], A[j * GLD + k], A[i * GLD + j]);
            }
            __syncwarp();
        }
        if (!ok) {
            for (int i = lane; i < n; i += 32) gterm[off + i] = 0.0;
            if (lane == 0) atomicAdd(&counters[CNT_GRAD_FAIL], 1);
            __syncwarp();
            continue;
        }
        // lambda = A^{-1} beta (in place in lam)
        for (int k = 0; k < n; ++k) {
            const double yk = lam[k] * A[k * GLD + k];
            __syncwarp();
            if (lane == (k & 31)) lam[k] = yk;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int i = lane + 32 * t;
                if (i > k && i < n) lam[i] = fma(-A[i * GLD + k], yk, lam[i]);
            }
            __syncwarp();
        }
        for (int k = n - 1; k >= 0; --k) {
            const double lk = lam[k] * A[k * GLD + k];
            __syncwarp();
            if (lane == (k & 31)) lam[k] = lk;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int i = lane + 32 * t;
                if (i < k) lam[i] = fma(-A[k * GLD + i], lk, lam[i]);
            }
            __syncwarp();
        }
        // K'_{jk} = kappa'(x_j - x_k) is odd in its argument: each pair once, both halves
        // stored (the factor in A is no longer needed)
        __syncwarp();
        for (int e = lane; e < n * (n - 1) / 2; e += 32) {
            int i, j;
            tri_index(e, i, j);          // (i, j), j <= i, of the (n-1)-triangle: pair (i + 1, j)
            ++i;
            const double v = g_kappa_prime(xl[i], xl[j], pv[i], pv[j], kp);
            A[i * GLD + j] = v;
            A[j * GLD + i] = -v;
        }
        for (int j = lane; j < n; j += 32) A[j * GLD + j] = 0.0;
        __syncwarp();
        // per node j (lanes own rows): -lambda_j kappa'(t_lj) - lambda_j (K'b)_j - b_j (K'lambda)_j
        for (int j = lane; j < n; j += 32) {
            double kb = 0.0, kl = 0.0;
            for (int k = 0; k < n; ++k) {
                const double kpjk = A[j * GLD + k];
                kb = fma(kpjk, bb[k], kb);
                kl = fma(kpjk, lam[k], kl);
            }
            const double tk = g_kappa_prime(tl, xl[j], pl, pv[j], kp);
            gterm[off + j] = -lam[j] * tk - lam[j] * kb - bb[j] * kl;
        }
        __syncwarp();
    }
}

// Per sorted node: dL/dx_j = sum of its terms over the columns of I(x_j).
__global__ void k_grad_gather(const double* __restrict__ gterm, const uint32_t* __restrict__ skey,
                              const int32_t* __restrict__ perm, const int32_t* __restrict__ col_start,
                              const int32_t* __restrict__ col_off, int N, int Ms, int m, double* __restrict__ gx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t key = skey[i];
    const int cell = (int)(key >> 1);
    const int first = cell - m + (int)(key & 1u);
    double acc = 0.0;
    for (int c = first; c <= cell + m; ++c) {
        int q = c;
        if (q < 0) q += Ms; else if (q >= Ms) q -= Ms;
        int pos = i - col_start[q];
        if (pos < 0) pos += N;
        acc += gterm[col_off[q] + pos];
    }
    gx[perm[i]] = acc;
}

}  // namespace

cudaError_t run_grad_nodes(Plan* p, const void* f, const void* w, double* gx, cudaStream_t s) {
    const int N = (int)p->N, Ms = (int)p->Ms;
    cudaError_t e = run_fft_forward<float>(p, w, s);     // gamma = F D w into p->grid
    if (e != cudaSuccess) return e;
    GradParams kp;
    kp.M = (double)p->M;
    kp.inv_Ms = 1.0 / (double)Ms;
    kp.sym = (p->kernel == INFFT_KERNEL_SYM);
    kp.diag = (kp.sym ? (double)(p->M - 1) : (double)p->M) / (double)Ms;
    {
        // kappa'_full(t) = -(1/M_sigma) sum_p (-1)^p (2 pi)^{2p+2} S_{2p+2} t^{2p+1} / (2p+1)!,
        // S_q = sum_{k=-M/2}^{M/2-1} k^q (the sym correction is added in the kernel)
        long double S[10] = {0};
        const long long half = p->M / 2;
        for (long long k = -half; k < half; ++k) {
            const long double k2 = (long double)k * (long double)k;
            long double pw = k2;
            for (int q = 0; q < 10; ++q) {
                S[q] += pw;          // k^{2q+2}
                pw *= k2;
            }
        }
        long double fact = 1.0L, tp = 4.0L * (long double)PI * (long double)PI;   // (2 pi)^{2p+2}
        for (int q = 0; q < 10; ++q) {
            if (q > 0) fact *= (long double)(2 * q) * (long double)(2 * q + 1);
            const long double sign = (q & 1) ? -1.0L : 1.0L;
            kp.cs[q] = (double)(-sign * tp * S[q] / (fact * (long double)Ms));
            tp *= 4.0L * (long double)PI * (long double)PI;
        }
    }
    {
        // pairs of a column are within (2m + 2)/M_sigma; the fourth terms of u cot u and
        // u^2/sin^2 u (2/945 u^6, 2/189 u^6) below 2^-56 let three terms stand
        const double u = PI * (double)(2 * p->m + 2) / (double)Ms;
        kp.short_series = (2.0 / 189.0) * u * u * u * u * u * u < std::ldexp(1.0, -56);
    }
    const KernelParams kk = make_kernel_params(p);
    const double mu = p->tau * kp.diag;
    if ((e = cudaMemsetAsync(p->counters + CNT_GRAD_FAIL, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    const int sms = p->sms;
    const size_t smem = (size_t)GW * (GN * GLD + 6 * GN) * sizeof(double);
    if ((e = cudaFuncSetAttribute(k_grad_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    launch_begin(p, "grad_cols", s);
    k_grad_cols<<<4 * sms, GW * 32, smem, s>>>(p->xs, p->phase, p->perm, p->col_start, p->col_count, p->col_off,
                                               p->w64, (const float2*)f, (const float2*)p->grid, N, Ms, kp, kk, mu,
                                               p->gterm, p->counters);
    launch_end(p, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    launch_begin(p, "grad_gather", s);
    k_grad_gather<<<(N + 255) / 256, 256, 0, s>>>(p->gterm, p->skey, p->perm, p->col_start, p->col_off, N, Ms,
                                                  p->m, gx);
    launch_end(p, s);
    return cudaGetLastError();
}
