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

// Programmatic dependent launch (sm_90+): a kernel launched with
// launch_pdl() may be scheduled while its predecessor in the stream is still
// running.  It must call griddep_wait() before it touches global memory that
// earlier stream work reads or writes; griddep_launch() lets the next kernel
// of the stream be scheduled early.
INFFT_D void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
INFFT_D void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Asynchronous global -> shared copies (cp.async): every copy of a thread is in
// flight at once; cp_async_wait_all() waits for this thread's copies, and a
// __syncthreads() after it publishes them to the CTA.
INFFT_D void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
INFFT_D void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
INFFT_D void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}
