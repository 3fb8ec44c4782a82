// Diagnostics: a measurement of this GPU's fp64 FMA throughput, the denominator of the
// fp64-bound precompute's roofline (the method itself has no counterpart of it).
#include "plan.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;     // independent FMA chains per thread

// Each thread advances PROBE_CHAINS independent recurrences a <- a * b + c for `iters`
// steps (2 flop each) and stores their sum, so nothing is dead code.  b < 1 keeps every
// value finite and normal.
__global__ void __launch_bounds__(PROBE_THREADS) k_fma64_probe(int64_t iters, double b, double c,
                                                              double* __restrict__ sink) {
    double a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    sink[(size_t)blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

}  // namespace

extern "C" infft_status infft_fp64_fma_probe(int64_t iters, double* sink, int64_t sink_len, double* flops,
                                             infft_stream_t stream) {
    if (iters < 1 || !sink || !flops) return set_error(INFFT_EINVAL, "iters >= 1, sink and flops are required");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_error(INFFT_ECUDA, "device query: %s", cudaGetErrorString(e));
    const int blocks = 8 * sms;   // 64 warps per SM
    const int64_t need = (int64_t)blocks * PROBE_THREADS;
    if (sink_len < need)
        return set_error(INFFT_EINVAL, "sink holds %lld doubles, the probe writes %lld", (long long)sink_len,
                         (long long)need);
    k_fma64_probe<<<blocks, PROBE_THREADS, 0, (cudaStream_t)stream>>>(iters, 0.999999, 1e-7, sink);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_error(INFFT_ECUDA, "launch: %s", cudaGetErrorString(e));
    count_launches(1);
    *flops = 2.0 * PROBE_CHAINS * (double)iters * (double)need;
    return INFFT_OK;
}

extern "C" int64_t infft_fp64_fma_probe_sink_len(void) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (int64_t)8 * sms * PROBE_THREADS;
}
