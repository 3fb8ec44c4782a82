// Length-M_sigma FFT with the diagonal D fused into its last pass.
//
// Adjoint direction (the inverse NFFT, eq:approx_ansatz2):
//   fhat_k = conj(d_k) * sum_{l} g_l exp(-2 pi i k l / M_sigma),  k = -M/2 .. M/2-1,
// with l = p - M_sigma/2, i.e. fhat_k = d_k (-1)^k DFT(g)[k mod M_sigma] (d_k real).
// Forward direction (the modified NFFT, Remark remark:ansatz2_adj):
//   g_l = sum_k exp(2 pi i k l / M_sigma) d_k fhat_k,
// i.e. g_p = sum_q Ghat_q exp(+2 pi i q p / M_sigma), Ghat_{k mod M_sigma} = (-1)^k d_k fhat_k.
// d_k = 1/M_sigma (kernel full); kernel sym sets d_{-M/2} = 0 (eq:matrix_D with
// Remark remark:Dirichlet_ansatz2).
//
// Transforms are radix-2 Stockham passes in shared memory (Govindaraju et al.,
// "High performance discrete Fourier transforms on graphics processors", SC 2008).
// M_sigma <= FFT_SMALL runs in one CTA; larger lengths use the four-step split
// M_sigma = N1 * N2 (p = N2 p1 + p2, k = k1 + N1 k2): pass A transforms over p1 at
// fixed p2 and applies the twiddle w^{p2 k1}; pass B transforms over p2 and writes
// the pruned, deconvolved output.  Twiddles come from sincospi on exactly reduced
// arguments.
#include <climits>
#include <mutex>

#include "plan.h"
#include "fft_r8.cuh"

namespace {

constexpr int FFT_THREADS = 256;
constexpr int FFT_SMALL = 2048;

template <typename T> INFFT_D cplx_t<T> czero() { return cmake((T)0, (T)0); }

// ---- single-CTA transform --------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_small_adjoint(const cplx_t<T>* __restrict__ g, cplx_t<T>* __restrict__ fhat, int logMs, int M, T inv_Ms,
                    int sym) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* a = (C*)smem_raw;
    const int Ms = 1 << logMs;
    C* b = a + Ms;
    for (int i = threadIdx.x; i < Ms; i += blockDim.x) a[i] = g[i];
    __syncthreads();
    C* res = smem_fft<T, -1>(a, b, logMs, 1);
    for (int kk = threadIdx.x; kk < M; kk += blockDim.x) {
        const int k = kk - M / 2;
        fhat[kk] = cscale(res[k & (Ms - 1)], deconv<T>(k, M, inv_Ms, sym));
    }
}

template <typename T>
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_small_forward(const cplx_t<T>* __restrict__ fhat, cplx_t<T>* __restrict__ g, int logMs, int M, T inv_Ms,
                    int sym) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* a = (C*)smem_raw;
    const int Ms = 1 << logMs;
    C* b = a + Ms;
    for (int q = threadIdx.x; q < Ms; q += blockDim.x) {
        const int k = bin_to_k(q, Ms, M);
        a[q] = (k == INT_MIN) ? czero<T>() : cscale(fhat[k + M / 2], deconv<T>(k, M, inv_Ms, sym));
    }
    __syncthreads();
    C* res = smem_fft<T, +1>(a, b, logMs, 1);
    for (int i = threadIdx.x; i < Ms; i += blockDim.x) g[i] = res[i];
}

// ---- four-step transform ---------------------------------------------------

// Pass A: CTA owns p2 in [p2_0, p2_0 + CA); transforms over p1 (length N1 = 2^log1),
// multiplies by w^{p2 k1} and stores Y[k1 * N2 + p2].  FORWARD_INPUT: the input
// is built from fhat (forward direction) instead of read from g.
template <typename T, int DIR, bool FORWARD_INPUT>
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_passA(const cplx_t<T>* __restrict__ in, cplx_t<T>* __restrict__ Y, int log1, int log2, int CA, int M,
            T inv_Ms, int sym) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N1 = 1 << log1, N2 = 1 << log2, Ms = N1 * N2;
    C* a = (C*)smem_raw;
    C* b = a + CA * N1;
    const int p2_0 = blockIdx.x * CA;
    for (int t = threadIdx.x; t < CA * N1; t += blockDim.x) {
        const int c = t % CA, p1 = t / CA;     // consecutive threads read consecutive p2
        const int q = (p1 << log2) + p2_0 + c;
        C v;
        if (FORWARD_INPUT) {
            const int k = bin_to_k(q, Ms, M);
            v = (k == INT_MIN) ? czero<T>() : cscale(in[k + M / 2], deconv<T>(k, M, inv_Ms, sym));
        } else {
            v = in[q];
        }
        a[c * N1 + p1] = v;
    }
    __syncthreads();
    C* res = smem_fft<T, DIR>(a, b, log1, CA);
    for (int t = threadIdx.x; t < CA * N1; t += blockDim.x) {
        const int c = t % CA, k1 = t / CA;
        const int p2 = p2_0 + c;
        const unsigned r = ((unsigned)p2 * (unsigned)k1) & (unsigned)(Ms - 1);   // exact reduction
        const C w = expipi((T)(DIR * 2) * (T)r / (T)Ms);
        Y[(k1 << log2) + p2] = cmul(res[c * N1 + k1], w);
    }
}

// Pass B: CTA owns k1 in [k1_0, k1_0 + CB); transforms rows Y[k1][.] of length
// N2 and writes X[k1 + N1 k2].  ADJOINT_OUTPUT: prune to the M central
// frequencies and apply (-1)^k d_k; otherwise store all M_sigma grid values.
template <typename T, int DIR, bool ADJOINT_OUTPUT>
__global__ void __launch_bounds__(FFT_THREADS)
k_fft_passB(const cplx_t<T>* __restrict__ Y, cplx_t<T>* __restrict__ out, int log1, int log2, int CB, int M,
            T inv_Ms, int sym) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N1 = 1 << log1, N2 = 1 << log2, Ms = N1 * N2;
    C* a = (C*)smem_raw;
    C* b = a + CB * N2;
    const int k1_0 = blockIdx.x * CB;
    for (int t = threadIdx.x; t < CB * N2; t += blockDim.x) a[t] = Y[((k1_0 + t / N2) << log2) + (t % N2)];
    __syncthreads();
    C* res = smem_fft<T, DIR>(a, b, log2, CB);
    for (int t = threadIdx.x; t < CB * N2; t += blockDim.x) {
        const int c = t % CB, k2 = t / CB;     // consecutive threads write consecutive q
        const int q = k1_0 + c + (k2 << log1);
        const C v = res[c * N2 + k2];
        if (ADJOINT_OUTPUT) {
            const int k = bin_to_k(q, Ms, M);
            if (k != INT_MIN) out[k + M / 2] = cscale(v, deconv<T>(k, M, inv_Ms, sym));
        } else {
            out[q] = v;
        }
    }
}

template <typename K> cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Launches both passes for a length-2^(log1+log2) grid; the pass B launch is
// programmatically dependent on pass A (and pass A on the spread before it).
cudaError_t fft_adjoint_r8(const float2* g, float2* work, float2* fhat, int logMs, int M, int sym, cudaStream_t s,
                           Plan* p, int K = 1) {
    const int log2 = logMs / 2, log1 = logMs - log2;
    const int Ms = 1 << logMs;
    const float inv_Ms = 1.0f / (float)Ms;
    const R8Shape a = r8_shape(log1, 1 << log2, K), b = r8_shape(log2, 1 << log1, K);
    void (*ka)(const float2*, float2*, int, int) = nullptr;
    void (*kb)(const float2*, float2*, int, int, int, float, int) = nullptr;
    switch (log1) {
        case 6: ka = k_fftA_r8<6>; break;
        case 7: ka = k_fftA_r8<7>; break;
        case 8: ka = k_fftA_r8<8>; break;
        case 9: ka = k_fftA_r8<9>; break;
        case 10: ka = k_fftA_r8<10>; break;
        case 11: ka = k_fftA_r8<11>; break;
        case 12: ka = k_fftA_r8<12>; break;
        default: return cudaErrorInvalidValue;
    }
    switch (log2) {
        case 6: kb = k_fftB_r8<6>; break;
        case 7: kb = k_fftB_r8<7>; break;
        case 8: kb = k_fftB_r8<8>; break;
        case 9: kb = k_fftB_r8<9>; break;
        case 10: kb = k_fftB_r8<10>; break;
        case 11: kb = k_fftB_r8<11>; break;
        case 12: kb = k_fftB_r8<12>; break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e;
    if ((e = allow_smem(ka, (size_t)a.smem)) != cudaSuccess) return e;
    if ((e = allow_smem(kb, (size_t)b.smem)) != cudaSuccess) return e;
    if (p) launch_begin(p, "fft_passA", s);
    e = launch_pdl(ka, dim3((1 << log2) / a.per_cta, K), dim3(a.per_cta * a.threads_per), (size_t)a.smem, s, g, work,
                   log2, a.per_cta);
    if (p) launch_end(p, s);
    if (e != cudaSuccess) return e;
    if (p) launch_begin(p, "fft_passB_deconv", s);
    e = launch_pdl(kb, dim3((1 << log1) / b.per_cta, K), dim3(b.per_cta * b.threads_per), (size_t)b.smem, s, work, fhat,
                   log1, b.per_cta, M, inv_Ms, sym);
    if (p) launch_end(p, s);
    return e;
}

// ---- the fp32 2-D transform of the tensor-product plan ------------------------
//
// fhat[k1 + M1/2][k2 + M2/2] = (-1)^(k1+k2) d_k sum_{a1, a2} g[a1][a2] e^{-2 pi i (k1 a1/Ms1 + k2 a2/Ms2)}
// (grid index a_t = l_t + Ms_t/2, so e^{-2 pi i k l/Ms} = (-1)^k e^{-2 pi i k a/Ms}): a row pass
// over a2 that keeps the M2 central k2, then a column pass over a1 for each kept k2.

// Rows: CTA owns grid rows a1 in [blockIdx.x CB, +CB) (thread t: row c = t / T2, j = t mod T2),
// transforms over a2 (length N2 = 2^LOG2) and stores Y[a1 M2 + k2 + M2/2] = (-1)^k2 value.
template <int LOG2>
__global__ void __launch_bounds__(512) k_fft2_rows_r8(const float2* __restrict__ g, float2* __restrict__ Y, int CB,
                                                      int M2) {
    constexpr int N2 = 1 << LOG2, T2 = N2 / 8, RS = N2 + N2 / 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tw = (float2*)smem_raw;
    const int t = threadIdx.x, c = t / T2, j = t % T2;
    float2* bufA = tw + N2 + 2 * c * RS;
    r8_twiddles<N2>(tw, t, blockDim.x);
    griddep_wait();
    griddep_launch();
    const int a1 = blockIdx.x * CB + c;
    float2 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = g[(a1 << LOG2) + j + r * T2];
    fft_r8<LOG2, -1>(v, bufA, bufA + RS, tw, j);
#pragma unroll
    for (int sl = 0; sl < 8; ++sl) {
        const int k2 = bin_to_k(r8_bin<LOG2>(j, sl), N2, M2);
        if (k2 != INT_MIN) Y[a1 * M2 + k2 + M2 / 2] = (k2 & 1) ? make_float2(-v[sl].x, -v[sl].y) : v[sl];
    }
}

// Columns: CTA owns kept columns kk in [blockIdx.x CA, +CA) (thread t: column c = t mod CA,
// j = t / CA), transforms Y[a1 M2 + kk] over a1 (length N1 = 2^LOG1) and stores
// fhat[(k1 + M1/2) M2 + kk] = (-1)^k1 d_k value (d_k = inv, 0 for kernel sym at k1 = -M1/2
// or k2 = -M2/2, i.e. kk = 0).
template <int LOG1>
__global__ void __launch_bounds__(512) k_fft2_cols_r8(const float2* __restrict__ Y, float2* __restrict__ fhat, int CA,
                                                      int M1, int M2, float inv, int sym) {
    constexpr int N1 = 1 << LOG1, T1 = N1 / 8, RS = N1 + N1 / 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tw = (float2*)smem_raw;
    const int t = threadIdx.x, c = t % CA, j = t / CA;
    float2* bufA = tw + N1 + 2 * c * RS;
    r8_twiddles<N1>(tw, t, blockDim.x);
    griddep_wait();
    griddep_launch();
    const int kk = blockIdx.x * CA + c;
    float2 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = Y[(j + r * T1) * M2 + kk];
    fft_r8<LOG1, -1>(v, bufA, bufA + RS, tw, j);
#pragma unroll
    for (int sl = 0; sl < 8; ++sl) {
        const int k1 = bin_to_k(r8_bin<LOG1>(j, sl), N1, M1);
        if (k1 == INT_MIN) continue;
        float d = (k1 & 1) ? -inv : inv;
        if (sym && (k1 == -M1 / 2 || kk == 0)) d = 0.0f;
        fhat[(k1 + M1 / 2) * M2 + kk] = make_float2(v[sl].x * d, v[sl].y * d);
    }
}

using RowsFn = void (*)(const float2*, float2*, int, int);
using ColsFn = void (*)(const float2*, float2*, int, int, int, float, int);

RowsFn pick_rows(int lg) {
    switch (lg) {
        case 6: return k_fft2_rows_r8<6>;
        case 7: return k_fft2_rows_r8<7>;
        case 8: return k_fft2_rows_r8<8>;
        case 9: return k_fft2_rows_r8<9>;
        case 10: return k_fft2_rows_r8<10>;
        case 11: return k_fft2_rows_r8<11>;
        default: return nullptr;
    }
}

ColsFn pick_cols(int lg) {
    switch (lg) {
        case 6: return k_fft2_cols_r8<6>;
        case 7: return k_fft2_cols_r8<7>;
        case 8: return k_fft2_cols_r8<8>;
        case 9: return k_fft2_cols_r8<9>;
        case 10: return k_fft2_cols_r8<10>;
        case 11: return k_fft2_cols_r8<11>;
        default: return nullptr;
    }
}

struct Split {
    int log1, log2, CA, CB;
};

template <typename T> Split choose_split(int logMs) {
    Split s;
    s.log2 = logMs / 2;
    s.log1 = logMs - s.log2;
    const int N1 = 1 << s.log1, N2 = 1 << s.log2;
    // aim for >= 128 CTAs per pass and <= 64 KB of shared memory per CTA
    const int cap_bytes = 64 * 1024;
    s.CA = N2 / 128; if (s.CA < 1) s.CA = 1; if (s.CA > 8) s.CA = 8;
    while (s.CA > 1 && 2 * s.CA * N1 * (int)sizeof(cplx_t<T>) > cap_bytes) s.CA >>= 1;
    s.CB = N1 / 128; if (s.CB < 1) s.CB = 1; if (s.CB > 8) s.CB = 8;
    while (s.CB > 1 && 2 * s.CB * N2 * (int)sizeof(cplx_t<T>) > cap_bytes) s.CB >>= 1;
    return s;
}

}  // namespace

// Launches pass B alone (the apply's second launch): rows of Y of length 2^log2, pruned and
// deconvolved output, programmatically dependent on the kernel before it.
cudaError_t fft_passB_r8(const float2* work, float2* fhat, int log1, int log2, int M, int sym, cudaStream_t s,
                         Plan* p, int K) {
    const int Ms = 1 << (log1 + log2);
    const float inv_Ms = 1.0f / (float)Ms;
    const R8Shape b = r8_shape(log2, 1 << log1, K);
    void (*kb)(const float2*, float2*, int, int, int, float, int) = nullptr;
    switch (log2) {
        case 6: kb = k_fftB_r8<6>; break;
        case 7: kb = k_fftB_r8<7>; break;
        case 8: kb = k_fftB_r8<8>; break;
        case 9: kb = k_fftB_r8<9>; break;
        case 10: kb = k_fftB_r8<10>; break;
        case 11: kb = k_fftB_r8<11>; break;
        case 12: kb = k_fftB_r8<12>; break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = allow_smem(kb, (size_t)b.smem);
    if (e != cudaSuccess) return e;
    if (p) launch_begin(p, "fft_passB_deconv", s);
    e = launch_pdl(kb, dim3((1 << log1) / b.per_cta, K), dim3(b.per_cta * b.threads_per), (size_t)b.smem, s, work,
                   fhat, log1, b.per_cta, M, inv_Ms, sym);
    if (p) launch_end(p, s);
    return e;
}


template <typename T>
cudaError_t run_fft_adjoint(Plan* p, void* fhat, cudaStream_t s) {
    using C = cplx_t<T>;
    const int Ms = (int)p->Ms, M = (int)p->M, logMs = p->logMs;
    const T inv_Ms = (T)1 / (T)Ms;
    const int sym = p->kernel == INFFT_KERNEL_SYM;
    cudaError_t e;
    if (Ms <= FFT_SMALL) {
        const size_t smem = 2 * (size_t)Ms * sizeof(C);
        if ((e = allow_smem(k_fft_small_adjoint<T>, smem)) != cudaSuccess) return e;
        launch_begin(p, sizeof(T) == 4 ? "fft_small" : "fft_small_z", s);
        k_fft_small_adjoint<T><<<1, FFT_THREADS, smem, s>>>((const C*)p->grid, (C*)fhat, logMs, M, inv_Ms, sym);
        launch_end(p, s);
        return cudaGetLastError();
    }
    if constexpr (sizeof(T) == 4) {
        if ((e = fft_adjoint_r8((const float2*)p->grid, (float2*)p->work, (float2*)fhat, logMs, M, sym, s, p)) !=
            cudaSuccess)
            return e;
        return cudaGetLastError();
    }
    const Split sp = choose_split<T>(logMs);
    const size_t smemA = 2 * (size_t)sp.CA * ((size_t)1 << sp.log1) * sizeof(C);
    const size_t smemB = 2 * (size_t)sp.CB * ((size_t)1 << sp.log2) * sizeof(C);
    if ((e = allow_smem(k_fft_passA<T, -1, false>, smemA)) != cudaSuccess) return e;
    if ((e = allow_smem(k_fft_passB<T, -1, true>, smemB)) != cudaSuccess) return e;
    launch_begin(p, sizeof(T) == 4 ? "fft_passA" : "fft_passA_z", s);
    k_fft_passA<T, -1, false><<<(1 << sp.log2) / sp.CA, FFT_THREADS, smemA, s>>>(
        (const C*)p->grid, (C*)p->work, sp.log1, sp.log2, sp.CA, M, inv_Ms, sym);
    launch_end(p, s);
    launch_begin(p, sizeof(T) == 4 ? "fft_passB_deconv" : "fft_passB_deconv_z", s);
    k_fft_passB<T, -1, true><<<(1 << sp.log1) / sp.CB, FFT_THREADS, smemB, s>>>(
        (const C*)p->work, (C*)fhat, sp.log1, sp.log2, sp.CB, M, inv_Ms, sym);
    launch_end(p, s);
    return cudaGetLastError();
}

// out_p = scale * sum_{k=-Mb/2}^{Mb/2-1} c_k in[k + Mb/2] exp(2 pi i k (p - M_sigma/2) / M_sigma),
// p = 0 .. M_sigma-1, for a band of Mb <= M_sigma frequencies (c_k = 0 only at k = -Mb/2 when
// sym); p->work is the four-step intermediate.
template <typename T>
cudaError_t fft_forward_on(Plan* p, const void* in, void* out, int Mb, T scale, int sym, cudaStream_t s) {
    using C = cplx_t<T>;
    const int Ms = (int)p->Ms, logMs = p->logMs;
    cudaError_t e;
    if (Ms <= FFT_SMALL) {
        const size_t smem = 2 * (size_t)Ms * sizeof(C);
        if ((e = allow_smem(k_fft_small_forward<T>, smem)) != cudaSuccess) return e;
        launch_begin(p, sizeof(T) == 4 ? "fft_small_fwd" : "fft_small_fwd_z", s);
        k_fft_small_forward<T><<<1, FFT_THREADS, smem, s>>>((const C*)in, (C*)out, logMs, Mb, scale, sym);
        launch_end(p, s);
        return cudaGetLastError();
    }
    const Split sp = choose_split<T>(logMs);
    const size_t smemA = 2 * (size_t)sp.CA * ((size_t)1 << sp.log1) * sizeof(C);
    const size_t smemB = 2 * (size_t)sp.CB * ((size_t)1 << sp.log2) * sizeof(C);
    if ((e = allow_smem(k_fft_passA<T, 1, true>, smemA)) != cudaSuccess) return e;
    if ((e = allow_smem(k_fft_passB<T, 1, false>, smemB)) != cudaSuccess) return e;
    launch_begin(p, sizeof(T) == 4 ? "fft_fwd_passA_deconv" : "fft_fwd_passA_deconv_z", s);
    k_fft_passA<T, 1, true><<<(1 << sp.log2) / sp.CA, FFT_THREADS, smemA, s>>>(
        (const C*)in, (C*)p->work, sp.log1, sp.log2, sp.CA, Mb, scale, sym);
    launch_end(p, s);
    launch_begin(p, sizeof(T) == 4 ? "fft_fwd_passB" : "fft_fwd_passB_z", s);
    k_fft_passB<T, 1, false><<<(1 << sp.log1) / sp.CB, FFT_THREADS, smemB, s>>>(
        (const C*)p->work, (C*)out, sp.log1, sp.log2, sp.CB, Mb, scale, sym);
    launch_end(p, s);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_fft_forward(Plan* p, const void* fhat, cudaStream_t s) {
    return fft_forward_on<T>(p, fhat, p->grid, (int)p->M, (T)1 / (T)p->Ms, p->kernel == INFFT_KERNEL_SYM, s);
}

cudaError_t run_fft_full_forward_z(Plan* p, const void* in, void* out, double scale, cudaStream_t s) {
    return fft_forward_on<double>(p, in, out, (int)p->Ms, scale, 0, s);
}

cudaError_t run_fft_forward_band_z(Plan* p, const void* in, void* out, cudaStream_t s) {
    return fft_forward_on<double>(p, in, out, (int)p->M, 1.0, 0, s);
}

// D^* F^* of K grids (grid: K x M_sigma, work: K x M_sigma, fhat: K x M), fp32, M_sigma > 2048.
cudaError_t run_fft_adjoint_many(Plan* p, const void* grid, void* work, void* fhat, int K, cudaStream_t s) {
    return fft_adjoint_r8((const float2*)grid, (float2*)work, (float2*)fhat, p->logMs, (int)p->M,
                          p->kernel == INFFT_KERNEL_SYM, s, p, K);
}

template cudaError_t run_fft_adjoint<float>(Plan*, void*, cudaStream_t);
template cudaError_t run_fft_adjoint<double>(Plan*, void*, cudaStream_t);
template cudaError_t run_fft_forward<float>(Plan*, const void*, cudaStream_t);
template cudaError_t run_fft_forward<double>(Plan*, const void*, cudaStream_t);

// ---- allocation-free entry point --------------------------------------------
//
// Callers that cannot allocate device memory at call time -- a process whose
// device memory is handed out entirely by its own pool allocator, or code that
// must not touch the allocator while another component is recording work -- get
// the pruned FFT with fused deconvolution (the last two steps of the inverse
// NFFT) without a plan.  Its only scratch, the four-step intermediate, lives in
// a file-scope device array that every GPU loading this library holds until the
// process exits.

namespace {

constexpr int NOALLOC_MAX_MS = 1 << 20;   // largest M_sigma (8 MiB of complex64 scratch)

__device__ __align__(256) float2 g_noalloc_scratch[NOALLOC_MAX_MS];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
struct NoallocSlot {
    void* ctx = nullptr;      // the context the address belongs to
    float2* addr = nullptr;
};
NoallocSlot g_noalloc_slot[NOALLOC_MAX_DEVICES];

// cuCtxGetCurrent, reached through the runtime's driver entry point query (the library
// links no driver library); nullptr when the query fails.
using CtxGetCurrentFn = int (*)(void**);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)ptr;
        else
            cudaGetLastError();
    }
    return fn;
}

// The device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in: the address must come from cudaGetSymbolAddress,
// looked up with the device current.  It is looked up on the first call on a device
// and again whenever the device's current context differs from the one it was taken
// in (after cudaDeviceReset the module is loaded anew and the array may move).
cudaError_t noalloc_scratch(int dev, float2** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    void* ctx = nullptr;
    if (CtxGetCurrentFn get = ctx_get_current()) {
        if (get(&ctx) != 0) ctx = nullptr;
    }
    NoallocSlot& slot = g_noalloc_slot[dev];
    if (!slot.addr || slot.ctx != ctx) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        slot.addr = (float2*)ptr;
        slot.ctx = ctx;
    }
    *out = slot.addr;
    return cudaSuccess;
}

bool on_device(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" infft_status infft_fft_deconv_noalloc(const float* grid, int64_t M, int64_t M_sigma, int kernel,
                                                 float* fhat, infft_stream_t stream) {
    if (!grid || !fhat) return set_error(INFFT_EINVAL, "grid and fhat must not be NULL");
    if (M < 2 || (M & 1)) return set_error(INFFT_EINVAL, "M must be even and >= 2 (got %lld)", (long long)M);
    if (M_sigma < M || M_sigma < 4 || (M_sigma & (M_sigma - 1)))
        return set_error(INFFT_EINVAL, "M_sigma must be a power of two >= max(M, 4) (got %lld)", (long long)M_sigma);
    if (M_sigma > NOALLOC_MAX_MS)
        return set_error(INFFT_EUNSUPPORTED, "M_sigma = %lld exceeds the %d of the allocation-free scratch",
                         (long long)M_sigma, NOALLOC_MAX_MS);
    if (kernel != INFFT_KERNEL_FULL && kernel != INFFT_KERNEL_SYM)
        return set_error(INFFT_EINVAL, "kernel must be INFFT_KERNEL_FULL or INFFT_KERNEL_SYM (got %d)", kernel);
    if (!on_device(grid) || !on_device(fhat))
        return set_error(INFFT_EINVAL, "grid and fhat must be device memory");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(INFFT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return set_error(INFFT_EUNSUPPORTED, "device %d", dev);
    float2* work = nullptr;
    if ((e = noalloc_scratch(dev, &work)) != cudaSuccess)
        return set_error(INFFT_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    const int Ms = (int)M_sigma, Mi = (int)M;
    int logMs = 0;
    while ((1 << logMs) < Ms) ++logMs;
    const float inv_Ms = 1.0f / (float)Ms;
    const int sym = kernel == INFFT_KERNEL_SYM;
    if (Ms <= FFT_SMALL) {
        const size_t smem = 2 * (size_t)Ms * sizeof(float2);
        if ((e = allow_smem(k_fft_small_adjoint<float>, smem)) != cudaSuccess)
            return set_error(INFFT_ECUDA, "%s", cudaGetErrorString(e));
        k_fft_small_adjoint<float><<<1, FFT_THREADS, smem, s>>>((const float2*)grid, (float2*)fhat, logMs, Mi,
                                                                 inv_Ms, sym);
        count_launches(1);
    } else {
        if ((e = fft_adjoint_r8((const float2*)grid, work, (float2*)fhat, logMs, Mi, sym, s, nullptr)) != cudaSuccess)
            return set_error(INFFT_ECUDA, "%s", cudaGetErrorString(e));
        count_launches(2);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return set_error(INFFT_ECUDA, "launch: %s", cudaGetErrorString(e));
    return INFFT_OK;
}

bool fft2d_r8_supported(int log1, int log2, int M2) {
    if (!pick_rows(log2) || !pick_cols(log1)) return false;
    const R8Shape b = r8_shape(log1, M2, 4);
    return M2 % b.per_cta == 0;
}

cudaError_t fft2d_adjoint_r8(const float2* g, float2* Y, float2* fhat, int log1, int log2, int M1, int M2, int sym,
                             cudaStream_t s) {
    RowsFn kr = pick_rows(log2);
    ColsFn kc = pick_cols(log1);
    if (!kr || !kc) return cudaErrorInvalidValue;
    const R8Shape a = r8_shape(log2, 1 << log1, 4), b = r8_shape(log1, M2, 4);
    if (M2 % b.per_cta) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = allow_smem(kr, (size_t)a.smem)) != cudaSuccess) return e;
    if ((e = allow_smem(kc, (size_t)b.smem)) != cudaSuccess) return e;
    const float inv = 1.0f / ((float)(1 << log1) * (float)(1 << log2));
    e = launch_pdl(kr, dim3((1 << log1) / a.per_cta), dim3(a.per_cta * a.threads_per), (size_t)a.smem, s, g, Y,
                   a.per_cta, M2);
    if (e != cudaSuccess) return e;
    e = launch_pdl(kc, dim3(M2 / b.per_cta), dim3(b.per_cta * b.threads_per), (size_t)b.smem, s, (const float2*)Y, fhat,
                   b.per_cta, M1, M2, inv, sym);
    count_launches(2);
    return e;
}
