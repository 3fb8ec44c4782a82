// Register-resident radix-8 Stockham transforms of the fp32 adjoint apply and the
// frequency bookkeeping of its pruned, deconvolved output (Sec. 3.2.2: fhat = D^* F^* g).
//
// Adjoint direction: fhat_k = conj(d_k) * sum_{l} g_l exp(-2 pi i k l / M_sigma),
// k = -M/2 .. M/2-1, with l = p - M_sigma/2, i.e. fhat_k = d_k (-1)^k DFT(g)[k mod M_sigma]
// (d_k real: 1/M_sigma, and 0 at k = -M/2 for kernel sym; eq:matrix_D with
// Remark remark:Dirichlet_ansatz2).  Large lengths use the four-step split
// M_sigma = N1 * N2 (p = N2 p1 + p2, k = k1 + N1 k2): pass A transforms over p1 at fixed p2
// and applies the twiddle w^{p2 k1}; pass B transforms over p2 and writes the pruned,
// deconvolved output.
#pragma once
#include <climits>

#include "fft_device.cuh"

namespace {

// Barriers of the transforms: the whole CTA, or the first NT threads (named barrier ID)
// when only part of the CTA runs the transform.
struct CtaSync {
    INFFT_D void operator()() const { __syncthreads(); }
};
template <int ID, int NT> struct NamedSync {
    INFFT_D void operator()() const { asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(NT) : "memory"); }
};

// frequency k of DFT bin q (or INT_MIN when q is pruned)
INFFT_D int bin_to_k(int q, int Ms, int M) {
    if (q < M / 2) return q;
    if (q >= Ms - M / 2) return q - Ms;
    return INT_MIN;
}

// (-1)^k d_k as a real factor (d_k = 1/M_sigma, 0 at k = -M/2 for kernel sym)
template <typename T> INFFT_D T deconv(int k, int M, T inv_Ms, int sym) {
    if (sym && k == -M / 2) return (T)0;
    return (k & 1) ? -inv_Ms : inv_Ms;
}

// ---- register-resident radix-8 Stockham transforms (fp32 adjoint apply) -----
//
// A length n = 2^LOGN transform is held by n/8 threads, 8 values each.  Every
// stage is a radix-R Stockham step (R = 8, and one final radix-4 or radix-2 step
// when LOGN is not a multiple of 3): butterfly jj reads a[jj + r n/R], multiplies
// value r by w^{r k n/(Ns R)} (k = jj mod Ns, w = e^{DIR 2 pi i/n}, Ns the length
// already transformed), runs a length-R DFT in registers and stores value r to
// a[(jj - k) R + k + r Ns].  The first stage takes its input from registers and
// the last leaves its output there: value slot s = b R + r of thread j holds bin
// j + b n/8 + r n/R.  Stages exchange values through shared memory (two
// buffers, one padding slot per 8 entries, so the stride-8 stores of the first
// stage hit distinct banks).  Twiddles come from a table of e^{DIR 2 pi i t/n}
// evaluated by sincospif on exact arguments.

INFFT_D int pad8(int i) { return i + (i >> 3); }

// One radix-R stage over this thread's butterflies jj = j + b n/8 (b < 8/R);
// dst == nullptr keeps the results in v (last stage).
template <int LOGN, int R, int DIR>
INFFT_D void r8_stage(float2 (&v)[8], const float2* src, float2* dst, const float2* tw, int j, int Ns) {
    constexpr int n = 1 << LOGN;
#pragma unroll
    for (int b = 0; b < 8 / R; ++b) {
        const int jj = j + b * (n / 8);
        float2* x = v + b * R;
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = src[pad8(jj + r * (n / R))];
        const int k = jj & (Ns - 1);
        const int step = k * (n / (Ns * R));
#pragma unroll
        for (int r = 1; r < R; ++r) x[r] = cmul(x[r], tw[r * step]);
        dft_r<DIR>(x, int_constant_tag<R>());
        if (dst) {
            const int base = (jj - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[pad8(base + r * Ns)] = x[r];
        }
    }
}

// bin held by value slot s of thread j after fft_r8<LOGN>
template <int LOGN> INFFT_D int r8_bin(int j, int s) {
    constexpr int n = 1 << LOGN, R = (LOGN % 3) ? (1 << (LOGN % 3)) : 8;
    return j + (s / R) * (n / 8) + (s % R) * (n / R);
}

// In: v[r] = x[j + r n/8].  Out: v[s] = X[r8_bin<LOGN>(j, s)].  bufA/bufB hold
// pad8(n) entries each; tw holds n twiddles.  Every thread that Sync waits for calls it
// (the whole CTA by default).
template <int LOGN, int DIR, typename Sync = CtaSync>
INFFT_D void fft_r8(float2 (&v)[8], float2* bufA, float2* bufB, const float2* tw, int j) {
    const Sync sync;
    constexpr int S8 = LOGN / 3, REM = LOGN % 3;
    static_assert(LOGN >= 6, "fft_r8 needs at least two stages");
    dft_r<DIR>(v, int_constant_tag<8>());
#pragma unroll
    for (int r = 0; r < 8; ++r) bufA[pad8(8 * j + r)] = v[r];
    float2* src = bufA;
    float2* dst = bufB;
    int Ns = 8;
#pragma unroll
    for (int st = 1; st < S8; ++st) {
        sync();
        const bool last = (st == S8 - 1) && REM == 0;
        r8_stage<LOGN, 8, DIR>(v, src, last ? nullptr : dst, tw, j, Ns);
        Ns *= 8;
        float2* t = src; src = dst; dst = t;
    }
    if (REM) {
        sync();
        r8_stage<LOGN, (REM ? (1 << REM) : 8), DIR>(v, src, nullptr, tw, j, Ns);
    }
}

// e^{-2 pi i t/n} for t < n (n a power of two >= 4): a quarter of the table by
// sincospif on exact arguments, the rest by exact quarter turns.
template <int n> INFFT_D void r8_twiddles(float2* tw, int t0, int stride) {
    for (int i = t0; i < n / 4; i += stride) {
        float sn, cs;
        sincospif((float)(-2 * i) / (float)n, &sn, &cs);
        tw[i] = make_float2(cs, sn);
        tw[i + n / 4] = make_float2(sn, -cs);          // * e^{-i pi/2}
        tw[i + n / 2] = make_float2(-cs, -sn);         // * e^{-i pi}
        tw[i + 3 * n / 4] = make_float2(-sn, cs);      // * e^{-3 i pi/2}
    }
}

// e^{-2 pi i t/Ms} for an integer t >= 0 (Ms a power of two), reduced exactly
INFFT_D float2 expm2pi_frac(int t, int Ms) {
    float sn, cs;
    sincospif((float)(-2 * (t & (Ms - 1))) / (float)Ms, &sn, &cs);
    return make_float2(cs, sn);
}

constexpr int R8_MIN_THREADS = 64;

// threads of one length-2^logn transform, transforms per CTA, shared bytes per CTA
struct R8Shape {
    int threads_per, per_cta, smem;
};

INFFT_HD R8Shape r8_shape(int logn, int count, int K = 1) {
    R8Shape s;
    s.threads_per = (1 << logn) / 8;
    s.per_cta = s.threads_per >= R8_MIN_THREADS ? 1 : R8_MIN_THREADS / s.threads_per;
    // several data vectors fill the GPU anyway: wider CTAs read whole 32-byte sectors
    // of the strided columns (4 consecutive complex64) and write longer output runs
    if (K >= 4 && s.threads_per < 256 && s.per_cta * s.threads_per < 256) s.per_cta = 256 / s.threads_per;
    if (s.per_cta > count) s.per_cta = count;
    const int n = 1 << logn;
    s.smem = (n + 2 * s.per_cta * (n + n / 8)) * (int)sizeof(float2);
    return s;
}

// Pass A of the fp32 adjoint four-step: CTA owns p2 in [blockIdx.x CA, +CA)
// (thread t: column c = t mod CA, j = t / CA); transforms g[p1 N2 + p2] over
// p1 (length N1 = 2^LOG1), multiplies bin k1 by w^{p2 k1} (w = e^{-2 pi i/M_sigma})
// and stores Y[k1 N2 + p2].
template <int LOG1>
__global__ void __launch_bounds__(512)
k_fftA_r8(const float2* __restrict__ g, float2* __restrict__ Y, int log2, int CA) {
    constexpr int N1 = 1 << LOG1, T1 = N1 / 8, RS = N1 + N1 / 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tw = (float2*)smem_raw;
    const int t = threadIdx.x, c = t % CA, j = t / CA;
    float2* bufA = tw + N1 + 2 * c * RS;
    r8_twiddles<N1>(tw, t, blockDim.x);
    griddep_wait();
    griddep_launch();
    const int p2 = blockIdx.x * CA + c;
    const int Ms = N1 << log2;
    g += (size_t)blockIdx.y * Ms;   // data vector blockIdx.y
    Y += (size_t)blockIdx.y * Ms;
    float2 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = g[((j + r * T1) << log2) + p2];
    fft_r8<LOG1, -1>(v, bufA, bufA + RS, tw, j);
    // w^{p2 k1} for the bins k1 = j + b N1/8 + r N1/R of this thread: three exact
    // evaluations and products (at most 8 roundings)
    constexpr int R = (LOG1 % 3) ? (1 << (LOG1 % 3)) : 8;
    const float2 wj = expm2pi_frac(p2 * j, Ms), wb = expm2pi_frac(p2 * (N1 / 8), Ms),
                 wr = expm2pi_frac(p2 * (N1 / R), Ms);
    float2 rowb = wj;
#pragma unroll
    for (int b = 0; b < 8 / R; ++b) {
        float2 w = rowb;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int s = b * R + r;
            Y[(r8_bin<LOG1>(j, s) << log2) + p2] = cmul(v[s], w);
            w = cmul(w, wr);
        }
        rowb = cmul(rowb, wb);
    }
}

// Pass B: CTA owns rows k1 in [blockIdx.x CB, +CB) (thread t: row c = t / T2,
// j = t mod T2); transforms Y[k1 N2 + p2] over p2 (length N2 = 2^LOG2) and writes
// bin q = k1 + N1 k2 pruned to the M central frequencies with (-1)^k d_k applied.
template <int LOG2>
__global__ void __launch_bounds__(512)
k_fftB_r8(const float2* __restrict__ Y, float2* __restrict__ fhat, int log1, int CB, int M, float inv_Ms,
          int sym) {
    constexpr int N2 = 1 << LOG2, T2 = N2 / 8, RS = N2 + N2 / 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tw = (float2*)smem_raw;
    const int t = threadIdx.x, c = t / T2, j = t % T2;
    float2* bufA = tw + N2 + 2 * c * RS;
    r8_twiddles<N2>(tw, t, blockDim.x);
    griddep_wait();
    griddep_launch();
    const int k1 = blockIdx.x * CB + c;
    const int Ms = N2 << log1;
    Y += (size_t)blockIdx.y * Ms;   // data vector blockIdx.y
    fhat += (size_t)blockIdx.y * M;
    float2 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = Y[(k1 << LOG2) + j + r * T2];
    fft_r8<LOG2, -1>(v, bufA, bufA + RS, tw, j);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int q = k1 + (r8_bin<LOG2>(j, s) << log1);
        const int k = bin_to_k(q, Ms, M);
        if (k != INT_MIN) fhat[k + M / 2] = cscale(v[s], deconv<float>(k, M, inv_Ms, sym));
    }
}

}  // namespace
