// Spreading g = B_opt^* f onto the oversampled grid (Sec. 3.2.2, the first factor
// of D^* F^* B_opt^* f) and its adjoint, the interpolation f = B_opt g (Remark
// remark:ansatz2_adj).  B_opt is stored column by column: the weights of grid
// point l are contiguous, aligned with the sorted nodes of I(l).
#include "plan.h"

namespace {

// One thread per grid point: a segmented gather, deterministic and atomic-free.
// In the fp32 path, "wide" columns (large ||b_l||_1, cancelling terms) use the
// fp64 weights and an fp64 accumulator; the fp64 path always does.
template <typename T>
__global__ void k_spread(const cplx_t<T>* __restrict__ f, const float* __restrict__ w32,
                         const double* __restrict__ w64, const uint8_t* __restrict__ wide,
                         const int32_t* __restrict__ perm, const int32_t* __restrict__ col_start,
                         const int32_t* __restrict__ col_count, const int32_t* __restrict__ col_off, int N,
                         int Ms, cplx_t<T>* __restrict__ g) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Ms) return;
    const int n = col_count[p], s = col_start[p], off = col_off[p];
    int q = s;
    if (sizeof(T) == 8 || wide[p]) {
        double re = 0, im = 0;
        for (int i = 0; i < n; ++i) {
            const double wi = w64[off + i];
            const cplx_t<T> v = f[perm[q]];
            re += wi * (double)v.x;
            im += wi * (double)v.y;
            if (++q == N) q = 0;
        }
        g[p] = cmake((T)re, (T)im);
    } else {
        float re = 0, im = 0;
        for (int i = 0; i < n; ++i) {
            const float wi = w32[off + i];
            const cplx_t<T> v = f[perm[q]];
            re += wi * (float)v.x;
            im += wi * (float)v.y;
            if (++q == N) q = 0;
        }
        g[p] = cmake((T)re, (T)im);
    }
}

// One thread per sorted node: gathers from the 2m (or 2m+1) grid points of I(x_j).
template <typename T>
__global__ void k_interp(const cplx_t<T>* __restrict__ g, const float* __restrict__ w32,
                         const double* __restrict__ w64, const uint8_t* __restrict__ wide,
                         const uint32_t* __restrict__ skey, const int32_t* __restrict__ perm,
                         const int32_t* __restrict__ col_start, const int32_t* __restrict__ col_off, int N,
                         int Ms, int m, cplx_t<T>* __restrict__ f) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t key = skey[i];
    const int cell = (int)(key >> 1);
    const int first = cell - m + (int)(key & 1u);   // integer nodes also meet cell - m
    float re32 = 0, im32 = 0;
    double re64 = 0, im64 = 0;
    for (int c = first; c <= cell + m; ++c) {
        int q = c;
        if (q < 0) q += Ms; else if (q >= Ms) q -= Ms;
        int pos = i - col_start[q];
        if (pos < 0) pos += N;
        const cplx_t<T> v = g[q];
        if (sizeof(T) == 8 || wide[q]) {
            const double wi = w64[col_off[q] + pos];
            re64 += wi * (double)v.x;
            im64 += wi * (double)v.y;
        } else {
            const float wi = w32[col_off[q] + pos];
            re32 += wi * (float)v.x;
            im32 += wi * (float)v.y;
        }
    }
    f[perm[i]] = cmake((T)(re64 + (double)re32), (T)(im64 + (double)im32));
}

}  // namespace

template <typename T>
cudaError_t run_spread(Plan* p, const void* f, cudaStream_t s) {
    const int Ms = (int)p->Ms;
    launch_begin(p, sizeof(T) == 4 ? "spread" : "spread_z", s);
    k_spread<T><<<(Ms + 255) / 256, 256, 0, s>>>((const cplx_t<T>*)f, p->w32, p->w64, p->wide, p->perm, p->col_start,
                                                  p->col_count, p->col_off, (int)p->N, Ms,
                                                  (cplx_t<T>*)p->grid);
    launch_end(p, s);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_interp(Plan* p, void* f, cudaStream_t s) {
    const int N = (int)p->N;
    launch_begin(p, sizeof(T) == 4 ? "interp" : "interp_z", s);
    k_interp<T><<<(N + 255) / 256, 256, 0, s>>>((const cplx_t<T>*)p->grid, p->w32, p->w64, p->wide, p->skey, p->perm,
                                                 p->col_start, p->col_off, N, (int)p->Ms, p->m,
                                                 (cplx_t<T>*)f);
    launch_end(p, s);
    return cudaGetLastError();
}

template cudaError_t run_spread<float>(Plan*, const void*, cudaStream_t);
template cudaError_t run_spread<double>(Plan*, const void*, cudaStream_t);
template cudaError_t run_interp<float>(Plan*, void*, cudaStream_t);
template cudaError_t run_interp<double>(Plan*, void*, cudaStream_t);
