// Device pieces of the FFT kernels.
//
// Register-level pieces: length-2, 4 and 8 DFTs of complex
// fp32 values held in registers, X_k = sum_r x_r e^{DIR 2 pi i r k / R}, output in
// natural order.
#pragma once
#include "common.cuh"

template <int R> struct int_constant_tag {};

template <int DIR> __device__ __forceinline__ static float2 mul_dir_i(float2 a) {   // a * (DIR i)
    return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int DIR> __device__ __forceinline__ static void dft_r(float2* x, int_constant_tag<2>) {
    const float2 a = x[0];
    x[0] = cadd(a, x[1]);
    x[1] = csub(a, x[1]);
}

template <int DIR> __device__ __forceinline__ static void dft_r(float2* x, int_constant_tag<4>) {
    const float2 a0 = cadd(x[0], x[2]), a1 = csub(x[0], x[2]);
    const float2 b0 = cadd(x[1], x[3]), b1 = mul_dir_i<DIR>(csub(x[1], x[3]));
    x[0] = cadd(a0, b0);
    x[2] = csub(a0, b0);
    x[1] = cadd(a1, b1);
    x[3] = csub(a1, b1);
}

template <int DIR> __device__ __forceinline__ static void dft_r(float2* x, int_constant_tag<8>) {
    float2 e[4] = {x[0], x[2], x[4], x[6]}, o[4] = {x[1], x[3], x[5], x[7]};
    dft_r<DIR>(e, int_constant_tag<4>());
    dft_r<DIR>(o, int_constant_tag<4>());
    const float h = 0.70710678118654752f;
    const float d = (float)DIR;
    o[1] = make_float2(h * (o[1].x - d * o[1].y), h * (o[1].y + d * o[1].x));   // * e^{DIR i pi/4}
    o[2] = mul_dir_i<DIR>(o[2]);                                                  // * e^{DIR i pi/2}
    o[3] = make_float2(-h * (o[3].x + d * o[3].y), h * (d * o[3].x - o[3].y));  // * e^{DIR 3 i pi/4}
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        x[k] = cadd(e[k], o[k]);
        x[k + 4] = csub(e[k], o[k]);
    }
}


// Batched radix-2 Stockham FFTs of length n = 2^logn in shared memory.  a holds
// `batch` transforms back to back; b is scratch of the same size.  Returns the
// buffer that holds the result.  DIR = -1: exp(-2 pi i ...), +1: exp(+2 pi i ...).
template <typename T, int DIR>
__device__ __forceinline__ static cplx_t<T>* smem_fft(cplx_t<T>* a, cplx_t<T>* b, int logn, int batch) {
    using C = cplx_t<T>;
    const int n = 1 << logn, half = n >> 1;
    const int total = batch * half;
    for (int Ns = 1; Ns < n; Ns <<= 1) {
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int bi = t >> (logn - 1), j = t & (half - 1);
            const C* src = a + bi * n;
            C* dst = b + bi * n;
            const int jm = j & (Ns - 1);
            C v0 = src[j], v1 = src[j + half];
            v1 = cmul(v1, expipi((T)(DIR * jm) / (T)Ns));
            const int d = ((j - jm) << 1) + jm;
            dst[d] = cadd(v0, v1);
            dst[d + Ns] = csub(v0, v1);
        }
        __syncthreads();
        C* tmp = a; a = b; b = tmp;
    }
    return a;
}

