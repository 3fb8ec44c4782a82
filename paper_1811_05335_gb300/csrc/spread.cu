// Spreading g = B_opt^* f onto the oversampled grid (Sec. 3.2.2, the first factor
// of D^* F^* B_opt^* f) and its adjoint, the interpolation f = B_opt g (Remark
// remark:ansatz2_adj).  B_opt is stored column by column: the weights of grid
// point l are contiguous, aligned with the sorted nodes of I(l).
#include "plan.h"
#include "spread_device.cuh"

namespace {

// Spreading in the precision of T (the fp64 apply; the fp32 apply uses k_spread_f32 or the
// fused kernel of apply.cu).  A CTA owns SPREAD_COLS consecutive grid points: their
// weights are one contiguous block of B_opt's storage and their nodes one contiguous
// (wrapping) range of sorted nodes, so both are staged in shared memory with coalesced
// loads before each thread sums its own column (fp32 staging only; fp64 reads directly).

template <typename T>
__global__ void __launch_bounds__(SPREAD_COLS)
k_spread(const cplx_t<T>* __restrict__ f, const float* __restrict__ w32, const double* __restrict__ w64,
         const float* __restrict__ wlo, const uint8_t* __restrict__ wide, const int32_t* __restrict__ perm,
         const int32_t* __restrict__ col_start,
         const int32_t* __restrict__ col_count, const int32_t* __restrict__ col_off, int N, int Ms,
         cplx_t<T>* __restrict__ g) {
    __shared__ __align__(16) float ws[SPREAD_WMAX];
    __shared__ cplx_t<T> fu[sizeof(T) == 4 ? SPREAD_UMAX : 1];
    const int p0 = blockIdx.x * SPREAD_COLS;
    const int p = p0 + threadIdx.x;
    const int plast = min(p0 + SPREAD_COLS, Ms) - 1;
    const bool live = p < Ms;
    const int n = live ? col_count[p] : 0;
    const int s = live ? col_start[p] : 0;
    const int off = live ? col_off[p] : 0;
    const bool wide_col = live && wide[p];
    // the block's weights [w0, w1) and nodes [S, S + U) (mod N)
    const int w0 = col_off[p0], w1 = col_off[plast + 1];
    const int S = col_start[p0];
    int U = 0;
    {
        int e = col_start[plast] + col_count[plast] - S;
        if (e < 0) e += N;
        U = e;
    }
    int r0 = s - S;
    if (r0 < 0) r0 += N;
    // every column's nodes must lie in the staged window (an empty first column need not bound it)
    const int inside = !live || n == 0 || (r0 + n <= U);
    const bool staged = __syncthreads_and(inside) && sizeof(T) == 4 && (w1 - w0) <= SPREAD_WMAX &&
                        U <= SPREAD_UMAX && U <= N;
    if (!staged) {
        if (live) g[p] = spread_direct<T>(f, w32, w64, wlo, wide_col, perm, n, s, off, N);
        return;
    }
    // weights: 16-byte vector loads of the aligned part, scalar edges
    {
        const int a0 = (w0 + 3) & ~3, a1 = w1 & ~3;
        if (a0 < a1) {
            const float4* src = (const float4*)(w32 + a0);
            for (int v = threadIdx.x; v < (a1 - a0) / 4; v += SPREAD_COLS) {
                const float4 t = src[v];
                const int d = a0 - w0 + 4 * v;
                ws[d] = t.x; ws[d + 1] = t.y; ws[d + 2] = t.z; ws[d + 3] = t.w;
            }
            for (int i = w0 + threadIdx.x; i < a0; i += SPREAD_COLS) ws[i - w0] = w32[i];
            for (int i = a1 + threadIdx.x; i < w1; i += SPREAD_COLS) ws[i - w0] = w32[i];
        } else {
            for (int i = w0 + threadIdx.x; i < w1; i += SPREAD_COLS) ws[i - w0] = w32[i];
        }
    }
    for (int q = threadIdx.x; q < U; q += SPREAD_COLS) {
        int gq = S + q;
        if (gq >= N) gq -= N;
        fu[q] = f[perm[gq]];
    }
    __syncthreads();
    if (!live) return;
    if (wide_col) {
        g[p] = spread_direct<T>(f, w32, w64, wlo, true, perm, n, s, off, N);
        return;
    }
    const float* wc = ws + (off - w0);
    float re = 0, im = 0;
    for (int i = 0; i < n; ++i) {
        const float wi = wc[i];
        const cplx_t<T> v = fu[r0 + i];
        re += wi * (float)v.x;
        im += wi * (float)v.y;
    }
    g[p] = cmake((T)re, (T)im);
}

// The fp32 spreading of the apply (one tile of SPREAD_COLS grid points per CTA),
// launched as a programmatically dependent kernel.
__global__ void __launch_bounds__(SPREAD_COLS)
k_spread_f32(const float2* __restrict__ f, const float* __restrict__ w32, const float* __restrict__ wlo,
             const uint8_t* __restrict__ wide, const int32_t* __restrict__ perm,
             const int32_t* __restrict__ col_start, const int32_t* __restrict__ col_count,
             const int32_t* __restrict__ col_off, int N, int Ms, float2* __restrict__ g) {
    __shared__ __align__(16) float ws[SPREAD_WMAX];
    __shared__ __align__(16) float2 fu[SPREAD_UMAX];
    griddep_wait();
    griddep_launch();
    // data vector blockIdx.y: f and g of vector k at k N and k M_sigma
    const int p0 = blockIdx.x * SPREAD_COLS;
    spread_tile_f32(f + (size_t)blockIdx.y * N, w32, wlo, wide, perm, col_start, col_count, col_off, N, p0,
                    min(p0 + SPREAD_COLS, Ms), g + (size_t)blockIdx.y * Ms, ws, fu);
}

// One thread per sorted node: gathers from the 2m (or 2m+1) grid points of I(x_j).
template <typename T>
__global__ void k_interp(const cplx_t<T>* __restrict__ g, const float* __restrict__ w32,
                         const double* __restrict__ w64, const float* __restrict__ wlo,
                         const uint8_t* __restrict__ wide,
                         const uint32_t* __restrict__ skey, const int32_t* __restrict__ perm,
                         const int32_t* __restrict__ col_start, const int32_t* __restrict__ col_off, int N,
                         int Ms, int m, cplx_t<T>* __restrict__ f) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t key = skey[i];
    const int cell = (int)(key >> 1);
    const int first = cell - m + (int)(key & 1u);   // integer nodes also meet cell - m
    if constexpr (sizeof(T) == 8) {
        double re = 0, im = 0;
        for (int c = first; c <= cell + m; ++c) {
            int q = c;
            if (q < 0) q += Ms; else if (q >= Ms) q -= Ms;
            int pos = i - col_start[q];
            if (pos < 0) pos += N;
            const cplx_t<T> v = g[q];
            const double wi = w64[col_off[q] + pos];
            re += wi * (double)v.x;
            im += wi * (double)v.y;
        }
        f[perm[i]] = cmake((T)re, (T)im);
    } else {
        // fp32 terms, and the terms of wide columns in float-float (ffsum.cuh)
        float re = 0, im = 0;
        FFSum acc;
        for (int c = first; c <= cell + m; ++c) {
            int q = c;
            if (q < 0) q += Ms; else if (q >= Ms) q -= Ms;
            int pos = i - col_start[q];
            if (pos < 0) pos += N;
            const float2 v = make_float2((float)g[q].x, (float)g[q].y);
            const int e = col_off[q] + pos;
            if (wide[q]) {
                acc.add(w32[e], wlo[e], v);
            } else {
                re = fmaf(w32[e], v.x, re);
                im = fmaf(w32[e], v.y, im);
            }
        }
        acc.add(1.0f, 0.0f, make_float2(re, im));
        const float2 r = acc.value();
        f[perm[i]] = cmake((T)r.x, (T)r.y);
    }
}

}  // namespace

template <typename T>
cudaError_t run_spread(Plan* p, const void* f, cudaStream_t s) {
    const int Ms = (int)p->Ms;
    launch_begin(p, sizeof(T) == 4 ? "spread" : "spread_z", s);
    const int blocks = (Ms + SPREAD_COLS - 1) / SPREAD_COLS;
    cudaError_t e = cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        e = launch_pdl(k_spread_f32, dim3(blocks), dim3(SPREAD_COLS), 0, s, (const float2*)f, p->w32, p->wlo,
                       p->wide, p->perm, p->col_start, p->col_count, p->col_off, (int)p->N, Ms, (float2*)p->grid);
    } else {
        k_spread<T><<<blocks, SPREAD_COLS, 0, s>>>((const cplx_t<T>*)f, p->w32, p->w64, p->wlo, p->wide, p->perm,
                                                   p->col_start, p->col_count, p->col_off, (int)p->N, Ms,
                                                   (cplx_t<T>*)p->grid);
    }
    launch_end(p, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_interp(Plan* p, void* f, cudaStream_t s) {
    const int N = (int)p->N;
    launch_begin(p, sizeof(T) == 4 ? "interp" : "interp_z", s);
    k_interp<T><<<(N + 255) / 256, 256, 0, s>>>((const cplx_t<T>*)p->grid, p->w32, p->w64, p->wlo, p->wide, p->skey,
                                                 p->perm,
                                                 p->col_start, p->col_off, N, (int)p->Ms, p->m,
                                                 (cplx_t<T>*)f);
    launch_end(p, s);
    return cudaGetLastError();
}

template cudaError_t run_spread<float>(Plan*, const void*, cudaStream_t);
template cudaError_t run_spread<double>(Plan*, const void*, cudaStream_t);
template cudaError_t run_interp<float>(Plan*, void*, cudaStream_t);
template cudaError_t run_interp<double>(Plan*, void*, cudaStream_t);

// K data vectors at once (f: K x N, grid: K x M_sigma).  A CTA stages its tile's
// weights and node indices once and then streams the K vectors' node windows
// through MANY_NB shared-memory buffers (the next MANY_NB - 1 vectors' values are in
// flight while the current one is summed).  A tile whose block does not fit takes
// the one-vector tile path per vector.
static constexpr int MANY_UMAX = SPREAD_UMAX / 2;   // node values per buffer
static constexpr int MANY_NB = 4;                   // buffers (prefetch depth MANY_NB - 1)
static constexpr size_t MANY_SMEM = SPREAD_WMAX * sizeof(float) + MANY_NB * MANY_UMAX * sizeof(float2);

static __global__ void __launch_bounds__(SPREAD_COLS, 3)
k_spread_many(const float2* __restrict__ f, int K, const float* __restrict__ w32, const float* __restrict__ wlo,
              const uint8_t* __restrict__ wide, const int32_t* __restrict__ perm,
              const int32_t* __restrict__ col_start, const int32_t* __restrict__ col_count,
              const int32_t* __restrict__ col_off, int N, int Ms, float2* __restrict__ g) {
    extern __shared__ __align__(16) unsigned char many_raw[];   // MANY_SMEM bytes
    float* ws = (float*)many_raw;                                  // SPREAD_WMAX
    float2* fu = (float2*)(many_raw + SPREAD_WMAX * sizeof(float)); // MANY_NB * MANY_UMAX
    griddep_wait();
    griddep_launch();
    const int p0 = blockIdx.x * SPREAD_COLS, p1 = min(p0 + SPREAD_COLS, Ms);
    const int p = p0 + threadIdx.x;
    const bool live = p < p1;
    const int n = live ? col_count[p] : 0;
    const int s = live ? col_start[p] : 0;
    const int off = live ? col_off[p] : 0;
    const bool wide_col = live && wide[p];
    const int w0 = col_off[p0], w1 = col_off[p1];
    const int S = col_start[p0];
    int U = col_start[p1 - 1] + col_count[p1 - 1] - S;
    if (U < 0) U += N;
    int r0 = s - S;
    if (r0 < 0) r0 += N;
    const int wb = w0 & ~3, we = (w1 + 3) & ~3;
    const int inside = !live || n == 0 || (r0 + n <= U);
    const bool staged = __syncthreads_and(inside) && (we - wb) <= SPREAD_WMAX && U <= MANY_UMAX && U <= N;
    if (!staged) {
        for (int k = 0; k < K; ++k) {
            spread_tile_f32(f + (size_t)k * N, w32, wlo, wide, perm, col_start, col_count, col_off, N, p0, p1,
                            g + (size_t)k * Ms, ws, fu);
            __syncthreads();
        }
        return;
    }
    for (int v = threadIdx.x; v < (we - wb) / 4; v += SPREAD_COLS) cp_async16(ws + 4 * v, w32 + wb + 4 * v);
    constexpr int UPT = MANY_UMAX / SPREAD_COLS;
    int pq[UPT];
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
        const int q = threadIdx.x + u * SPREAD_COLS;
        int gq = S + q;
        if (gq >= N) gq -= N;
        pq[u] = q < U ? perm[gq] : 0;
    }
    auto issue = [&](int k) {
        const float2* fk = f + (size_t)k * N;
        float2* dst = fu + (k % MANY_NB) * MANY_UMAX;
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
            const int q = threadIdx.x + u * SPREAD_COLS;
            if (q < U) cp_async8(dst + q, fk + pq[u]);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    for (int k = 0; k < MANY_NB - 1 && k < K; ++k) issue(k);   // the first with the weights
    for (int k = 0; k < K; ++k) {
        if (k + MANY_NB - 1 < K) issue(k + MANY_NB - 1);
        // groups still allowed in flight: those of vectors k+1 .. min(K-1, k+MANY_NB-1)
        const int ahead = min(K - 1 - k, MANY_NB - 1);
        if (ahead >= 3) asm volatile("cp.async.wait_group 3;" ::: "memory");
        else if (ahead == 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
        else if (ahead == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
        else asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        if (live) {
            float2* gk = g + (size_t)k * Ms;
            if (wide_col) {
                gk[p] = spread_direct<float>(f + (size_t)k * N, w32, nullptr, wlo, true, perm, n, s, off, N);
            } else {
                // walk the column from a lane-dependent start (see spread_tile_f32)
                const float* wc = ws + (off - wb);
                const float2* fc = fu + (k % MANY_NB) * MANY_UMAX + r0;
                float re = 0, im = 0;
                int j = n ? (int)(threadIdx.x & 31) % n : 0;
                for (int i = 0; i < n; ++i) {
                    const float wi = wc[j];
                    const float2 v = fc[j];
                    re = fmaf(wi, v.x, re);
                    im = fmaf(wi, v.y, im);
                    j = (j + 1 == n) ? 0 : j + 1;
                }
                gk[p] = make_float2(re, im);
            }
        }
        __syncthreads();   // buffer k % MANY_NB is refilled for vector k + MANY_NB
    }
}

cudaError_t run_spread_many(Plan* p, const void* f, void* grid, int K, cudaStream_t s) {
    const int Ms = (int)p->Ms;
    cudaError_t e = cudaFuncSetAttribute(k_spread_many, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MANY_SMEM);
    if (e != cudaSuccess) return e;
    launch_begin(p, "spread_many", s);
    e = launch_pdl(k_spread_many, dim3((Ms + SPREAD_COLS - 1) / SPREAD_COLS), dim3(SPREAD_COLS), MANY_SMEM, s,
                   (const float2*)f, K, p->w32, p->wlo, p->wide, p->perm, p->col_start, p->col_count, p->col_off,
                   (int)p->N, Ms, (float2*)grid);
    launch_end(p, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
