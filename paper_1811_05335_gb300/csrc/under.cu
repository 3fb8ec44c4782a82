// Underdetermined case (Sec. 3.2.1): B_opt from one least-squares problem per
// node x_j,
//     min over real b of ||K_j b - M e_j||^2 + mu_j ||b||^2          (eq:opt_ansatz1)
// with K_j = (kappa(x_h - l/M_sigma))_{h = 1..N, l in I(x_j)} (eq:matrix_Kj; the
// Dirichlet choice of Remark remark:Dirichlet_ansatz1 makes kappa the kernel of the
// overdetermined case), mu_j = tau * (mean diagonal entry of Re K_j^* K_j), and the
// estimate f_check = (1/M) D^* F^* B_opt^* f (eq:approx_ansatz1).
//
// The normal matrix sums over all N nodes.  With the node moments
// mu_n = sum_h exp(2 pi i n x_h), |n| < M, it depends only on grid-point pairs:
//     S(l, l') = sum_h conj(kappa(x_h - l/Ms)) kappa(x_h - l'/Ms)
//              = Ms^{-2} sum_n mu_n Q(n, l - l') exp(-2 pi i n l'/Ms),
//     Q(n, d)  = sum over kept k with k + n kept of exp(2 pi i k d/Ms)
//              = exp(-i pi d (n + 1)/Ms) sin(pi (M - |n|) d/Ms) / sin(pi d/Ms)  (full),
// the sym kernel removing the term k = -M/2 (n >= 0) or k = -M/2 - n (n < 0).  For
// each offset d = 0 .. 2m one full-length FFT gives S(l' + d, l') at every grid
// point l'; a node's Gram entries are then table reads, its right-hand side is
// M Re kappa(x_j - l/Ms) in closed form, and its (2m+1)-unknown system is solved
// by the thread tier's register Cholesky.  Work: O(N M) fp64 for the moments,
// 2m+1 FFTs of length Ms, O(m^3) per node.
//
// The coefficients are stored divided by M in the column layout of the
// overdetermined case (column l, position of node j in I(l)), so the same spread,
// FFT and D give f_check, and the same interpolation gives (1/M) B_opt F D h, the
// inverse adjoint estimate of Remark remark:ansatz1_adj.
#include <algorithm>

#include "lsq_device.cuh"

namespace {

constexpr int MOM_RUN = 32;        // consecutive frequencies n per thread
constexpr int MOM_THREADS = 128;
constexpr int MOM_CHUNKS_MAX = 64; // node chunks (partial sums per frequency)

// part[c * M + n] = sum over the nodes h of chunk c of exp(2 pi i n x_h), n = 0 .. M-1.
// A thread owns MOM_RUN consecutive n; exp(2 pi i n0 x_h) comes from an exactly
// reduced sincospi, the following n by multiplying with exp(2 pi i x_h).
__global__ void __launch_bounds__(MOM_THREADS)
k_moments(const double* __restrict__ xs, const double2* __restrict__ step, int N, int M, int chunk,
          double2* __restrict__ part) {
    const int n0 = (blockIdx.x * MOM_THREADS + threadIdx.x) * MOM_RUN;
    const int c = blockIdx.y;
    const int h0 = c * chunk, h1 = min(N, h0 + chunk);
    double re[MOM_RUN], im[MOM_RUN];
#pragma unroll
    for (int k = 0; k < MOM_RUN; ++k) re[k] = im[k] = 0.0;
    if (n0 < M) {
        for (int h = h0; h < h1; ++h) {
            const double2 z0 = phase_of(2.0 * (double)n0, xs[h]);    // (sin, cos)(2 pi n0 x_h)
            const double2 w = step[h];                                // (sin, cos)(2 pi x_h)
            double zr = z0.y, zi = z0.x;
#pragma unroll
            for (int k = 0; k < MOM_RUN; ++k) {
                re[k] += zr;
                im[k] += zi;
                const double t = fma(zr, w.y, -zi * w.x);
                zi = fma(zr, w.x, zi * w.y);
                zr = t;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < MOM_RUN; ++k)
        if (n0 + k < M) part[(size_t)c * M + n0 + k] = make_double2(re[k], im[k]);
}

__global__ void k_moment_steps(const double* __restrict__ xs, int N, double2* __restrict__ step) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h < N) step[h] = phase_of(2.0, xs[h]);
}

// mu_n = sum_c part[c][n] in chunk order (deterministic).
__global__ void k_moments_reduce(const double2* __restrict__ part, int chunks, int M, double2* __restrict__ mom) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= M) return;
    double r = 0.0, i = 0.0;
    for (int c = 0; c < chunks; ++c) {
        const double2 v = part[(size_t)c * M + n];
        r += v.x;
        i += v.y;
    }
    mom[n] = make_double2(r, i);
}

// (sin, cos)(pi a / Ms) for an integer a, reduced exactly modulo 2 Ms (Ms a power of two).
INFFT_D double2 sincos_frac(long long a, int Ms) {
    const long long P = 2LL * Ms;
    long long r = a % P;
    if (r < 0) r += P;
    double s, c;
    sincospi((double)r / (double)Ms, &s, &c);
    return make_double2(s, c);
}

// FFT input of offset d: in[k + Ms/2] = sum over n = -k (mod Ms), |n| < M, of mu_n Q(n, d).
__global__ void k_gram_input(const double2* __restrict__ mom, int M, int Ms, int d, int sym, double inv_sin_d,
                             double2* __restrict__ in) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Ms) return;
    const int k = q - Ms / 2;
    double ar = 0.0, ai = 0.0;
    for (int w = -1; w <= 1; ++w) {
        const long long n = -(long long)k + (long long)w * Ms;
        if (n <= -M || n >= M) continue;
        const int an = (int)(n < 0 ? -n : n);
        double2 mu = mom[an];
        if (n < 0) mu.y = -mu.y;                       // mu_{-n} = conj(mu_n)
        double qr, qi;
        if (d == 0) {
            qr = (double)(M - an);
            qi = 0.0;
        } else {
            const double2 ph = sincos_frac(-(long long)d * (n + 1), Ms);               // exp(-i pi d (n+1)/Ms)
            const double mag = sincos_frac((long long)(M - an) * d, Ms).x * inv_sin_d;  // Dirichlet ratio
            qr = ph.y * mag;
            qi = ph.x * mag;
        }
        if (sym) {
            // drop k = -M/2 (n >= 0) or k + n = -M/2 (n < 0): exp(2 pi i k d / Ms) at that k
            const long long kk = (n >= 0) ? -(long long)(M / 2) : -(long long)(M / 2) - n;
            const double2 e = sincos_frac(2 * kk * d, Ms);
            qr -= e.y;
            qi -= e.x;
        }
        ar += mu.x * qr - mu.y * qi;
        ai += mu.x * qi + mu.y * qr;
    }
    in[q] = make_double2(ar, ai);
}

// Per node (sorted position i): Re S on its run of grid points, right-hand side,
// Cholesky, coefficients into the column layout (divided by M), objective.
template <int NMAX, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_under_lsq(const double* __restrict__ xs, const double2* __restrict__ ph, const uint32_t* __restrict__ skey,
            const int32_t* __restrict__ perm, const int32_t* __restrict__ col_start,
            const int32_t* __restrict__ col_count, const int32_t* __restrict__ col_off,
            const double2* __restrict__ S, int N, int Ms, int m, KernelParams kp, double tau,
            double* __restrict__ w64, float* __restrict__ w32, double* __restrict__ Jout,
            int32_t* __restrict__ counters) {
    extern __shared__ double lsq_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* T = lsq_smem + (size_t)wid * 32 * (NMAX * (NMAX + 1) / 2) + lane;   // T[e * 32]
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t key = skey[i];
    const int cell = (int)(key >> 1);
    const int p0 = cell - m + (int)(key & 1u);      // first column: ceil(u) - m (storage index)
    const int n = 2 * m + 1 - (int)(key & 1u);
    if (n > NMAX) {
        atomicAdd(&counters[CNT_UNSUPPORTED], 1);
        return;
    }
    int pa[NMAX];
#pragma unroll
    for (int a = 0; a < NMAX; ++a) {
        int q = p0 + a;
        q %= Ms;
        if (q < 0) q += Ms;
        pa[a] = q;
    }
    const double x = xs[i];
    const double2 px = ph[i];
    double v[NMAX], dsum = 0.0;
#pragma unroll
    for (int a = 0; a < NMAX; ++a) {
        if (a < n) {
            const double t = col_t(pa[a], Ms);
            v[a] = kp.M * re_kappa(x, t, px, phase_of(kp.M, t), kp);
            dsum += S[pa[a]].x;
        }
    }
    double mu = tau * dsum / (double)n;
    bool ok = false;
    double ysq = 0.0, b[NMAX];
    for (int attempt = 0; attempt < 3 && !ok; ++attempt) {
#pragma unroll
        for (int a = 0; a < NMAX; ++a) {
            if (a < n) {
#pragma unroll
                for (int c = 0; c <= a; ++c)
                    T[(trow(a) + c) * 32] = S[(size_t)(a - c) * Ms + pa[c]].x + (a == c ? mu : 0.0);
                b[a] = v[a];
            }
        }
        ok = chol_solve<NMAX>(T, n, b, ysq);
        if (!ok) mu *= 1e3;
    }
    const double invM = 1.0 / kp.M;
    double bsq = 0.0;
#pragma unroll
    for (int a = 0; a < NMAX; ++a) {
        if (a < n) {
            const int q = pa[a];
            int pos = i - col_start[q];
            if (pos < 0) pos += N;
            const double wv = ok ? b[a] * invM : 0.0;
            if (pos < col_count[q]) {
                store_b(w64, w32, kp.wlo, col_off[q] + pos, wv);
            } else {
                atomicAdd(&counters[CNT_UNSUPPORTED], 1);   // the pattern and the key disagree
            }
            bsq = fma(b[a], b[a], bsq);
        }
    }
    const double M2 = kp.M * kp.M;
    // J_j = ||K_j b - M e_j||^2 = M^2 - (M r).b - mu ||b||^2 at the regularised optimum
    Jout[perm[i]] = ok ? M2 - ysq - mu * bsq : M2;
    if (!ok || mu != tau * dsum / (double)n) atomicAdd(&counters[CNT_FALLBACK], 1);
}

// wide[p] = ||column p of B_opt / M||_1 > WIDE_COLUMN_L1 (fp64 spreading of that column).
__global__ void k_under_wide(const int32_t* __restrict__ col_count, const int32_t* __restrict__ col_off,
                             const double* __restrict__ w64, int Ms, uint8_t* __restrict__ wide) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Ms) return;
    const int off = col_off[p], n = col_count[p];
    double s = 0.0;
    for (int q = 0; q < n; ++q) s += fabs(w64[off + q]);
    wide[p] = s > WIDE_COLUMN_L1;
}

inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

template <int NMAX, int WARPS>
cudaError_t launch_under_lsq(Plan* p, const KernelParams& kp, cudaStream_t s) {
    const size_t smem = (size_t)WARPS * 32 * (NMAX * (NMAX + 1) / 2) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_under_lsq<NMAX, WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    launch_begin(p, "under_lsq", s);
    k_under_lsq<NMAX, WARPS><<<blocks_for(p->N, WARPS * 32), WARPS * 32, smem, s>>>(
        p->xs, p->phase, p->skey, p->perm, p->col_start, p->col_count, p->col_off, (const double2*)p->under_S,
        (int)p->N, (int)p->Ms, p->m, kp, p->tau, p->w64, p->w32, p->J, p->counters);
    launch_end(p, s);
    return cudaGetLastError();
}

}  // namespace

int under_moment_chunks(int64_t N) {
    int64_t c = (N + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(MOM_CHUNKS_MAX, c));
}

cudaError_t run_precompute_under(Plan* p, cudaStream_t s) {
    const int N = (int)p->N, M = (int)p->M, Ms = (int)p->Ms, m = p->m;
    const KernelParams kp = make_kernel_params(p);
    cudaError_t e = cudaMemsetAsync(p->counters + CNT_FALLBACK, 0, 2 * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p->w64, 0, (size_t)p->nnz_cap * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p->w32, 0, (size_t)p->nnz_cap * sizeof(float), s)) != cudaSuccess) return e;

    // node moments mu_n, n = 0 .. M-1
    double2* step = (double2*)p->under_step;
    double2* part = (double2*)p->under_part;
    double2* mom = (double2*)p->under_mom;
    const int chunks = under_moment_chunks(N);
    const int chunk = (N + chunks - 1) / chunks;
    launch_begin(p, "under_steps", s);
    k_moment_steps<<<blocks_for(N, 256), 256, 0, s>>>(p->xs, N, step);
    launch_end(p, s);
    const int runs = (M + MOM_RUN - 1) / MOM_RUN;
    launch_begin(p, "under_moments", s);
    k_moments<<<dim3(blocks_for(runs, MOM_THREADS), chunks), MOM_THREADS, 0, s>>>(p->xs, step, N, M, chunk, part);
    launch_end(p, s);
    launch_begin(p, "under_moments_reduce", s);
    k_moments_reduce<<<blocks_for(M, 256), 256, 0, s>>>(part, chunks, M, mom);
    launch_end(p, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    // S(l' + d, l') for d = 0 .. 2m: one full-length fp64 FFT each
    const int sym = p->kernel == INFFT_KERNEL_SYM;
    const double scale = 1.0 / ((double)Ms * (double)Ms);
    double2* S = (double2*)p->under_S;
    for (int d = 0; d <= 2 * m; ++d) {
        const double inv_sin_d = d ? 1.0 / sin(3.141592653589793238462643383279502884 * (double)d / (double)Ms) : 0.0;
        launch_begin(p, "under_gram_input", s);
        k_gram_input<<<blocks_for(Ms, 256), 256, 0, s>>>(mom, M, Ms, d, sym, inv_sin_d, (double2*)p->grid);
        launch_end(p, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = run_fft_full_forward_z(p, p->grid, S + (size_t)d * Ms, scale, s)) != cudaSuccess) return e;
    }

    // per-node systems
    if (2 * m + 1 <= 9) e = launch_under_lsq<9, 8>(p, kp, s);
    else e = launch_under_lsq<UNDER_NMAX, 4>(p, kp, s);
    if (e != cudaSuccess) return e;
    launch_begin(p, "under_wide", s);
    k_under_wide<<<blocks_for(Ms, 256), 256, 0, s>>>(p->col_count, p->col_off, p->w64, Ms, p->wide);
    launch_end(p, s);
    return cudaGetLastError();
}
