// Device helpers shared by the kernels of the GB300 iNFFT library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define INFFT_HD __host__ __device__ __forceinline__
#define INFFT_D __device__ __forceinline__

template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using cplx_t = typename cplx<T>::type;

INFFT_HD float2 cmake(float r, float i) { return make_float2(r, i); }
INFFT_HD double2 cmake(double r, double i) { return make_double2(r, i); }
template <typename C> INFFT_HD C cadd(C a, C b) { C c; c.x = a.x + b.x; c.y = a.y + b.y; return c; }
template <typename C> INFFT_HD C csub(C a, C b) { C c; c.x = a.x - b.x; c.y = a.y - b.y; return c; }
template <typename C> INFFT_HD C cmul(C a, C b) {
    C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
template <typename C, typename T> INFFT_HD C cscale(C a, T s) { C c; c.x = a.x * s; c.y = a.y * s; return c; }

// e^{i pi t} for a real t given exactly (sincospi keeps the argument exact).
INFFT_D float2 expipi(float t) { float s, c; sincospif(t, &s, &c); return make_float2(c, s); }
INFFT_D double2 expipi(double t) { double s, c; sincospi(t, &s, &c); return make_double2(c, s); }

INFFT_D unsigned lanemask_lt() { unsigned r; asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(r)); return r; }
