// Spreading g = B_opt^* f onto the grid for one tile of grid points (Sec. 3.2.2),
// shared by the single-problem and the batched apply.  B_opt is stored column
// by column: the weights of grid point l are contiguous, aligned with the sorted
// nodes of I(l).
#pragma once
#include "plan.h"
#include "ffsum.cuh"

namespace {

constexpr int SPREAD_COLS = 256;
constexpr int SPREAD_WMAX = 8192;     // staged weights per CTA (32 KB)
constexpr int SPREAD_UMAX = 2048;     // staged node values per CTA (16 KB)

// g_l of one column by direct loads: fp64 weights and accumulation for T = double; fp32 for
// T = float, float-float (w32 + wlo, ffsum.cuh) for wide columns.
template <typename T>
INFFT_D cplx_t<T> spread_direct(const cplx_t<T>* __restrict__ f, const float* __restrict__ w32,
                                const double* __restrict__ w64, const float* __restrict__ wlo, bool wide_col,
                                const int32_t* __restrict__ perm, int n, int s, int off, int N) {
    int q = s;
    if constexpr (sizeof(T) == 8) {
        double re = 0, im = 0;
        for (int i = 0; i < n; ++i) {
            const double wi = w64[off + i];
            const cplx_t<T> v = f[perm[q]];
            re += wi * (double)v.x;
            im += wi * (double)v.y;
            if (++q == N) q = 0;
        }
        return cmake((T)re, (T)im);
    } else {
        if (wide_col) {
            FFSum acc;
            for (int i = 0; i < n; ++i) {
                acc.add(w32[off + i], wlo[off + i], f[perm[q]]);
                if (++q == N) q = 0;
            }
            return acc.value();
        }
        float re = 0, im = 0;
        for (int i = 0; i < n; ++i) {
            const float wi = w32[off + i];
            const cplx_t<T> v = f[perm[q]];
            re += wi * (float)v.x;
            im += wi * (float)v.y;
            if (++q == N) q = 0;
        }
        return cmake((T)re, (T)im);
    }
}

// Spreads grid points [p0, p1) whose weights [w0, w1) do not fit a staging buffer
// (clustered nodes): the CTA (COLS threads) walks the entries in storage order, COLS at a
// time (coalesced weight and index loads); each thread follows its entry's column
// with a running pointer over the tile's offsets, a warp-level segmented sum
// combines neighbouring entries of one column and the segment's last lane adds it
// to the column's sum in shared memory.  Wide columns (float-float) are summed per
// thread afterwards.  iw: 2 COLS + 1 ints, gs: COLS float2 of shared
// memory.  Every thread of the CTA calls it.
template <int COLS = SPREAD_COLS>
INFFT_D void spread_tile_segmented(const float2* __restrict__ f, const float* __restrict__ w32,
                                   const float* __restrict__ wlo, const uint8_t* __restrict__ wide,
                                   const int32_t* __restrict__ perm, const int32_t* __restrict__ col_start,
                                   const int32_t* __restrict__ col_off, int N, int p0, int p1, int w0, int w1,
                                   float2* __restrict__ g, int* iw, float2* gs) {
    int* offs = iw;                         // ncols + 1 weight offsets
    int* cst = offs + COLS + 1;      // ncols node starts
    const int ncols = p1 - p0;
    for (int c = threadIdx.x; c <= ncols; c += COLS) {
        offs[c] = col_off[p0 + c];
        if (c < ncols) {
            cst[c] = col_start[p0 + c];
            gs[c] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int c = 0;
    for (int base = w0; base < w1; base += COLS) {
        const int e = base + threadIdx.x;
        const bool act = e < w1;
        float2 v = make_float2(0.f, 0.f);
        if (act) {
            while (offs[c + 1] <= e) ++c;
            if (!wide[p0 + c]) {
                int r = cst[c] + (e - offs[c]);
                if (r >= N) r -= N;
                const float2 fv = f[perm[r]];
                const float wi = w32[e];
                v = make_float2(wi * fv.x, wi * fv.y);
            }
        }
        const int key = act ? c : -1 - lane;     // inactive lanes form their own segments
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float tx = __shfl_up_sync(0xffffffffu, v.x, o);
            const float ty = __shfl_up_sync(0xffffffffu, v.y, o);
            const int tk = __shfl_up_sync(0xffffffffu, key, o);
            if (lane >= o && tk == key) { v.x += tx; v.y += ty; }
        }
        const int nk = __shfl_down_sync(0xffffffffu, key, 1);
        if (act && (lane == 31 || nk != key)) {
            atomicAdd(&gs[c].x, v.x);
            atomicAdd(&gs[c].y, v.y);
        }
    }
    __syncthreads();
    const int p = p0 + threadIdx.x;
    if (p < p1) {
        if (wide[p]) g[p] = spread_direct<float>(f, w32, nullptr, wlo, true, perm, col_off[p + 1] - col_off[p], col_start[p],
                                                  col_off[p], N);
        else g[p] = gs[threadIdx.x];
    }
}

// Spreads grid points [p0, p1) (p1 - p0 <= SPREAD_COLS) of a problem with Ms grid points
// into g (indexed by grid point): the tile's weights [w0, w1) move to shared
// memory by 16-byte asynchronous copies of the 16-byte aligned span around them,
// the node indices of the window come to registers and the node values follow by
// 8-byte asynchronous copies, so every load of the tile is in flight at once.
// Columns with large ||b_l||_1 spread in float-float; a tile whose block does not
// fit the staging buffers falls back to direct loads.  One thread per grid point;
// every thread of the CTA calls it.
constexpr int SPREAD_UPT = SPREAD_UMAX / SPREAD_COLS;   // staged node values per thread

INFFT_D void spread_tile_f32(const float2* __restrict__ f, const float* __restrict__ w32,
                             const float* __restrict__ wlo, const uint8_t* __restrict__ wide,
                             const int32_t* __restrict__ perm, const int32_t* __restrict__ col_start,
                             const int32_t* __restrict__ col_count, const int32_t* __restrict__ col_off, int N,
                             int p0, int p1, float2* __restrict__ g, float* ws, float2* fu) {
    const int p = p0 + threadIdx.x;
    const int plast = p1 - 1;
    const bool live = p < p1;
    const int n = live ? col_count[p] : 0;
    const int s = live ? col_start[p] : 0;
    const int off = live ? col_off[p] : 0;
    const bool wide_col = live && wide[p];
    const int w0 = col_off[p0], w1 = col_off[plast + 1];
    const int S = col_start[p0];
    int U = col_start[plast] + col_count[plast] - S;
    if (U < 0) U += N;
    int r0 = s - S;
    if (r0 < 0) r0 += N;
    const int wb = w0 & ~3, we = (w1 + 3) & ~3;
    const int inside = !live || n == 0 || (r0 + n <= U);
    const bool staged = __syncthreads_and(inside) && (we - wb) <= SPREAD_WMAX && U <= SPREAD_UMAX && U <= N;
    if (!staged) {
        spread_tile_segmented(f, w32, wlo, wide, perm, col_start, col_off, N, p0, p1, w0, w1, g, (int*)ws, fu);
        return;
    }
    for (int v = threadIdx.x; v < (we - wb) / 4; v += SPREAD_COLS) cp_async16(ws + 4 * v, w32 + wb + 4 * v);
    int pq[SPREAD_UPT];
#pragma unroll
    for (int u = 0; u < SPREAD_UPT; ++u) {
        const int q = threadIdx.x + u * SPREAD_COLS;
        int gq = S + q;
        if (gq >= N) gq -= N;
        pq[u] = q < U ? perm[gq] : 0;
    }
#pragma unroll
    for (int u = 0; u < SPREAD_UPT; ++u) {
        const int q = threadIdx.x + u * SPREAD_COLS;
        if (q < U) cp_async8(fu + q, f + pq[u]);
    }
    cp_async_wait_all();
    __syncthreads();
    if (!live) return;
    if (wide_col) {
        g[p] = spread_direct<float>(f, w32, nullptr, wlo, true, perm, n, s, off, N);
        return;
    }
    // Neighbouring threads' columns start about |I(l)| weights (and N/M_sigma nodes)
    // apart in shared memory, so walking every column from its start would put a
    // warp's accesses on a few banks; each thread starts its walk at its own lane
    // (mod n) instead, which spreads the accesses over the banks.
    const float* wc = ws + (off - wb);
    const float2* fc = fu + r0;
    float re = 0, im = 0;
    int k = n ? (int)(threadIdx.x & 31) % n : 0;
    for (int i = 0; i < n; ++i) {
        const float wi = wc[k];
        const float2 v = fc[k];
        re = fmaf(wi, v.x, re);
        im = fmaf(wi, v.y, im);
        k = (k + 1 == n) ? 0 : k + 1;
    }
    g[p] = make_float2(re, im);
}

}  // namespace
