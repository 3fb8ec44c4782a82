// The pattern step: index sets I(l) of eq:set_l as ranges of sorted nodes.
//
// A node with u = fl(M_sigma x) meets grid point l iff ceil(u) - m <= l <= floor(u) + m
// (mod M_sigma).  With cell b = floor(u) and the flag "u is an integer", the nodes of
// column l are: every node of cells l-m .. l+m-1, plus the integer nodes of cell l+m.
// Sorting the nodes by key = 2*cell + (u is not an integer) therefore turns every
// I(l) into one contiguous key range [2(l-m), 2(l+m)] that wraps modulo M_sigma.
//
// The sort is a stable LSD radix sort (8-bit digits): equal keys keep the caller's
// node order, so the whole pattern -- and every later result -- is deterministic.
#include "plan.h"

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;                       // keys per thread per tile
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;    // 2048 keys per tile
constexpr int RS_BINS = 256;

__global__ void k_node_keys(const double* __restrict__ x, int N, int Ms, uint32_t* __restrict__ key,
                            int32_t* __restrict__ val, int32_t* __restrict__ counters) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double xj = x[j];
    bool ok = isfinite(xj) && xj >= -0.5 && xj < 0.5;
    if (!ok) {
        atomicAdd(&counters[CNT_BAD_NODES], 1);
        xj = 0.0;   // keeps the pattern in range; the plan reports the bad node
    }
    double u = __dmul_rn((double)Ms, xj);   // one rounded product, never contracted
    double fb = floor(u);
    int exact = (u == fb);
    long long cell = (long long)fb + Ms / 2;  // in [0, Ms]; u may round up to Ms/2
    if (cell >= Ms) cell -= Ms;
    if (cell < 0) cell += Ms;
    key[j] = (uint32_t)(2 * cell + (exact ? 0 : 1));
    val[j] = j;
}

__global__ void k_rs_hist(const uint32_t* __restrict__ keys, int n, int shift, uint32_t* __restrict__ hist,
                          int tiles) {
    __shared__ uint32_t cnt[RS_BINS];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * RS_TILE;
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        int e = base + i * RS_THREADS + threadIdx.x;
        if (e < n) atomicAdd(&cnt[(keys[e] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];   // digit-major
}

// Stable scatter: warp w owns items [w*256, w*256+256) of the tile and walks them
// in 8 rounds of 32 consecutive keys; ranks among equal digits come from
// __match_any_sync, so the order inside a digit follows the input order.
__global__ void k_rs_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin, int n,
                             int shift, const uint32_t* __restrict__ hist, int tiles,
                             uint32_t* __restrict__ kout, int32_t* __restrict__ vout) {
    __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int base = blockIdx.x * RS_TILE + w * (RS_ITEMS * 32);
    uint32_t k[RS_ITEMS];
    int32_t v[RS_ITEMS];
    uint32_t local[RS_ITEMS];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        int e = base + r * 32 + lane;
        bool valid = e < n;
        k[r] = valid ? kin[e] : 0u;
        v[r] = valid ? vin[e] : 0;
        uint32_t d = valid ? ((k[r] >> shift) & 0xFF) : RS_BINS;   // invalid lanes share a dummy digit
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = (d < RS_BINS) ? wcnt[w][d] : 0u;
        local[r] = before + __popc(peers & lt);
        __syncwarp();
        if (d < RS_BINS && (peers & lt) == 0) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // exclusive scan over warps, per digit (one thread per digit)
        uint32_t run = 0;
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            uint32_t t = wcnt[ww][threadIdx.x];
            wcnt[ww][threadIdx.x] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        int e = base + r * 32 + lane;
        if (e < n) {
            uint32_t d = (k[r] >> shift) & 0xFF;
            uint32_t pos = hist[d * tiles + blockIdx.x] + wcnt[w][d] + local[r];
            kout[pos] = k[r];
            vout[pos] = v[r];
        }
    }
}

// Exclusive scan of n int32 values in two passes over blocks of SCAN_CHUNK: the
// first reduces each block, the second adds the prefix of the block sums and
// scans the block.  out may alias in; out has n + 1 entries, out[n] = total.
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

INFFT_D int32_t block_sum(int32_t v, int32_t* red) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int32_t t = 0;
    for (int w = 0; w < SCAN_THREADS / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const int32_t* __restrict__ in, int n,
                                                              int32_t* __restrict__ sums) {
    __shared__ int32_t red[SCAN_THREADS / 32];
    const int b0 = blockIdx.x * SCAN_CHUNK;
    int32_t s = 0;
    for (int i = threadIdx.x; i < SCAN_CHUNK; i += SCAN_THREADS)
        if (b0 + i < n) s += in[b0 + i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) sums[blockIdx.x] = s;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const int32_t* in, int32_t* out, int n,
                                                             const int32_t* __restrict__ sums) {
    __shared__ int32_t red[SCAN_THREADS / 32];
    __shared__ int32_t wsum[SCAN_THREADS / 32];
    int32_t before = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += SCAN_THREADS) before += sums[b];
    before = block_sum(before, red);
    const int b0 = blockIdx.x * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t loc = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (b0 + i < n) ? in[b0 + i] : 0;
        loc += v[i];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t inc = loc;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int32_t wpre = 0;
    for (int ww = 0; ww < w; ++ww) wpre += wsum[ww];
    int32_t run = before + wpre + inc - loc;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (b0 + i < n) out[b0 + i] = run;
        run += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = run;
}

__global__ void k_gather_x(const double* __restrict__ x, const int32_t* __restrict__ perm, int N,
                           double* __restrict__ xs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) xs[i] = x[perm[i]];
}

INFFT_D int lower_bound_u32(const uint32_t* __restrict__ a, int n, uint32_t v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_col_ranges(const uint32_t* __restrict__ skey, int N, int Ms, int m,
                             int32_t* __restrict__ start, int32_t* __restrict__ count,
                             int32_t* __restrict__ counters) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Ms) return;
    int lo = p - m; if (lo < 0) lo += Ms;
    int hi = p + m; if (hi >= Ms) hi -= Ms;
    uint32_t klo = 2u * (uint32_t)lo, khi = 2u * (uint32_t)hi + 1u;   // keys [klo, khi)
    int a = lower_bound_u32(skey, N, klo);
    int b = lower_bound_u32(skey, N, khi);
    int c = (klo < khi) ? (b - a) : (N - a) + b;
    start[p] = (a == N) ? 0 : a;
    count[p] = c;
    if (c == 0) atomicAdd(&counters[CNT_EMPTY], 1);
    atomicMax(&counters[CNT_MAX_COLUMN], c);
}

inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t run_exclusive_scan(Plan* p, const int32_t* in, int32_t* out, int n, cudaStream_t s) {
    const int nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK > 0 ? (n + SCAN_CHUNK - 1) / SCAN_CHUNK : 1;
    launch_begin(p, "scan_reduce", s);
    k_scan_reduce<<<nb, SCAN_THREADS, 0, s>>>(in, n, p->scan_sums);
    launch_end(p, s);
    launch_begin(p, "scan_apply", s);
    k_scan_apply<<<nb, SCAN_THREADS, 0, s>>>(in, out, n, p->scan_sums);
    launch_end(p, s);
    return cudaGetLastError();
}

cudaError_t run_pattern(Plan* p, cudaStream_t s) {
    const int N = (int)p->N, Ms = (int)p->Ms;
    cudaError_t e = cudaMemsetAsync(p->counters, 0, CNT_N * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;

    launch_begin(p, "node_keys", s);
    k_node_keys<<<blocks_for(N, 256), 256, 0, s>>>(p->x, N, Ms, p->keys[0], p->vals[0], p->counters);
    launch_end(p, s);

    const int tiles = blocks_for(N, RS_TILE);
    const int passes = (p->key_bits + 7) / 8;
    for (int pass = 0; pass < passes; ++pass) {
        const int in = pass & 1, out = in ^ 1, shift = 8 * pass;
        launch_begin(p, "radix_hist", s);
        k_rs_hist<<<tiles, RS_THREADS, 0, s>>>(p->keys[in], N, shift, p->hist, tiles);
        launch_end(p, s);
        e = run_exclusive_scan(p, (const int32_t*)p->hist, (int32_t*)p->hist, RS_BINS * tiles, s);
        if (e != cudaSuccess) return e;
        launch_begin(p, "radix_scatter", s);
        k_rs_scatter<<<tiles, RS_THREADS, 0, s>>>(p->keys[in], p->vals[in], N, shift, p->hist, tiles,
                                                   p->keys[out], p->vals[out]);
        launch_end(p, s);
    }
    launch_begin(p, "gather_x", s);
    k_gather_x<<<blocks_for(N, 256), 256, 0, s>>>(p->x, p->perm, N, p->xs);
    launch_end(p, s);

    launch_begin(p, "col_ranges", s);
    k_col_ranges<<<blocks_for(Ms, 256), 256, 0, s>>>(p->skey, N, Ms, p->m, p->col_start, p->col_count,
                                                     p->counters);
    launch_end(p, s);
    return run_exclusive_scan(p, p->col_count, p->col_off, Ms, s);
}
