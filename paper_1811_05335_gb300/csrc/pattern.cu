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

// Exclusive scan of n int32 values by one block (out may alias in; out has n+1
// entries and out[n] receives the total).
__global__ void k_scan_single(const int32_t* in, int32_t* out, int n) {
    __shared__ int32_t wsum[32];
    const int T = blockDim.x;
    const int chunk = (n + T - 1) / T;
    const int b = min(n, threadIdx.x * chunk), e = min(n, b + chunk);
    int32_t s = 0;
    for (int i = b; i < e; ++i) s += in[i];
    // block-wide exclusive scan of s
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int32_t ws = (lane < (T >> 5)) ? wsum[lane] : 0;
        int32_t wi = ws;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < (T >> 5)) wsum[lane] = wi - ws;
    }
    __syncthreads();
    int32_t run = wsum[w] + inc - s;
    for (int i = b; i < e; ++i) {
        int32_t t = in[i];
        out[i] = run;
        run += t;
    }
    if (threadIdx.x == T - 1) out[n] = run;
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
    launch_begin(p, "scan", s);
    k_scan_single<<<1, 1024, 0, s>>>(in, out, n);
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
