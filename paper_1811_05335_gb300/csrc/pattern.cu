// The pattern step: index sets I(l) of eq:set_l as ranges of sorted nodes.
//
// A node with u = fl(M_sigma x) meets grid point l iff ceil(u) - m <= l <= floor(u) + m
// (mod M_sigma).  With cell b = floor(u) and the flag "u is an integer", the nodes of
// column l are: every node of cells l-m .. l+m-1, plus the integer nodes of cell l+m.
// Sorting the nodes by key = 2*cell + (u is not an integer) therefore turns every
// I(l) into one contiguous key range [2(l-m), 2(l+m)] that wraps modulo M_sigma.
//
// The sort is a counting sort over the 2 M_sigma keys: a histogram, its exclusive
// scan (the bucket offsets, which also give every column's range directly), an
// atomic scatter, and a fix-up that orders each bucket by the caller's node index,
// so the result -- and every later result -- is deterministic.  A last pass
// gathers the sorted nodes and their phases (sin, cos)(pi M x) used by the
// precompute.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "plan.h"

namespace {

constexpr int SMALL_BUCKET = 32;   // buckets up to this size are ordered by one thread

INFFT_D uint32_t node_key(double xj, int Ms) {
    double u = __dmul_rn((double)Ms, xj);   // one rounded product, never contracted
    double fb = floor(u);
    int exact = (u == fb);
    long long cell = (long long)fb + Ms / 2;  // in [0, Ms]; u may round up to Ms/2
    if (cell >= Ms) cell -= Ms;
    if (cell < 0) cell += Ms;
    return (uint32_t)(2 * cell + (exact ? 0 : 1));
}

INFFT_D double checked_node(const double* __restrict__ x, int j) {
    const double xj = x[j];
    return (isfinite(xj) && xj >= -0.5 && xj < 0.5) ? xj : 0.0;   // bad nodes are counted in k_bucket_count
}

__global__ void k_bucket_count(const double* __restrict__ x, int N, int Ms, int32_t* __restrict__ bucket,
                               int32_t* __restrict__ counters) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double xj = x[j];
    if (!(isfinite(xj) && xj >= -0.5 && xj < 0.5)) atomicAdd(&counters[CNT_BAD_NODES], 1);
    atomicAdd(&bucket[node_key(checked_node(x, j), Ms)], 1);
}

__global__ void k_bucket_scatter(const double* __restrict__ x, int N, int Ms, const int32_t* __restrict__ bucket,
                                 int32_t* __restrict__ cursor, int32_t* __restrict__ perm,
                                 uint32_t* __restrict__ skey) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const uint32_t key = node_key(checked_node(x, j), Ms);
    const int pos = bucket[key] + atomicAdd(&cursor[key], 1);
    perm[pos] = j;
    skey[pos] = key;
}

// (sin, cos)(pi k / 1024) for k = -1024 .. 1024 at k + 1024, filled once per device
// (phase_table_init) from long double evaluations rounded to double.
constexpr int PHASE_TAB_HALF = 1024;
__device__ double2 g_phase_tab[2 * PHASE_TAB_HALF + 1];

// (sin, cos)(pi M z) with M z reduced modulo 2 exactly: M z = p + e with
// p = fl(M z) and e = fma(M, z, -p); p - 2 rint(p/2) is exact.  The angle
// a = r + e in [-1, 1] is split as k/1024 + d (d exact, |d| <= 1/2048): the table
// gives (sin, cos)(pi k/1024), short Taylor series (sin z = z - z^3/6 + z^5/120,
// cos z = 1 - z^2/2 + z^4/24 at |z| <= pi/2048, dropped terms below 1e-20
// relative) give (sin, cos)(pi d), and the angle addition joins them.
INFFT_D double2 node_phase(double M, double z) {
    const double p = M * z;
    const double e = fma(M, z, -p);
    const double r = p - 2.0 * rint(0.5 * p);
    const double a = r + e;
    const double kf = fmin(fmax(rint(a * (double)PHASE_TAB_HALF), -(double)PHASE_TAB_HALF), (double)PHASE_TAB_HALF);
    const double d = fma(kf, -1.0 / (double)PHASE_TAB_HALF, a);
    const double zz = 3.141592653589793238462643383279502884 * d;
    const double z2 = zz * zz;
    const double sd = zz * fma(z2, fma(z2, 1.0 / 120.0, -1.0 / 6.0), 1.0);
    const double cd = fma(z2, fma(z2, 1.0 / 24.0, -0.5), 1.0);
    const double2 t = g_phase_tab[(int)kf + PHASE_TAB_HALF];   // (sin, cos)(pi k/1024)
    return make_double2(fma(t.x, cd, t.y * sd), fma(t.y, cd, -(t.x * sd)));
}

// Per sorted node: its position and its phase (sin, cos)(pi M x).
__global__ void k_gather_nodes(const double* __restrict__ x, const int32_t* __restrict__ perm, int N, double M,
                               double* __restrict__ xs, double2* __restrict__ ph) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double xi = checked_node(x, perm[i]);
    xs[i] = xi;
    ph[i] = node_phase(M, xi);
}

// One thread per bucket: small buckets are ordered by caller index (insertion
// sort), larger ones are queued for k_bigseg_fixup.
__global__ void k_bucket_fixup(const int32_t* __restrict__ bucket, int nkeys, int32_t* __restrict__ perm,
                               int32_t* __restrict__ seg_list, int32_t* __restrict__ counters) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nkeys) return;
    const int s0 = bucket[b], s1 = bucket[b + 1], k = s1 - s0;
    if (k == 0) return;
    if (k > SMALL_BUCKET) {
        seg_list[atomicAdd(&counters[CNT_BIG_SEGMENTS], 1)] = b;
        return;
    }
    for (int i = s0 + 1; i < s1; ++i) {
        const int v = perm[i];
        int q = i - 1;
        while (q >= s0 && perm[q] > v) {
            perm[q + 1] = perm[q];
            --q;
        }
        perm[q + 1] = v;
    }
}

// One CTA per large bucket: each element's final position is its rank among the
// bucket's (distinct) caller indices; ranks are counted, written to tmp, copied back.
__global__ void k_bigseg_fixup(const int32_t* __restrict__ seg_list, const int32_t* __restrict__ counters,
                               const int32_t* __restrict__ bucket, int32_t* __restrict__ perm,
                               int32_t* __restrict__ tmp) {
    const int total = counters[CNT_BIG_SEGMENTS];
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int b = seg_list[it];
        const int s0 = bucket[b], s1 = bucket[b + 1], k = s1 - s0;
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            const int v = perm[s0 + i];
            int rank = 0;
            for (int q = 0; q < k; ++q) rank += perm[s0 + q] < v;
            tmp[s0 + rank] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < k; i += blockDim.x) perm[s0 + i] = tmp[s0 + i];
        __syncthreads();
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

// Column l (storage p) holds the keys [2(p-m), 2(p+m)] (mod 2 M_sigma): its range of
// sorted nodes starts at the offset of the first key and ends before the offset of
// the key after the last; the range wraps when the key interval does.
__global__ void k_col_ranges(const int32_t* __restrict__ bucket, int N, int Ms, int m, int32_t* __restrict__ start,
                             int32_t* __restrict__ count, int32_t* __restrict__ counters) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Ms) return;
    int lo = p - m; if (lo < 0) lo += Ms;
    int hi = p + m; if (hi >= Ms) hi -= Ms;
    const int klo = 2 * lo, khi = 2 * hi + 1;     // keys [klo, khi)
    const int a = bucket[klo], b = bucket[khi];
    const int c = (klo < khi) ? (b - a) : (N - a) + b;
    start[p] = (a == N) ? 0 : a;
    count[p] = c;
    if (c == 0) atomicAdd(&counters[CNT_EMPTY], 1);
    atomicMax(&counters[CNT_MAX_COLUMN], c);
}

inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t run_exclusive_scan(Plan* p, const int32_t* in, int32_t* out, int n, cudaStream_t s) {
    const int nb = n > 0 ? (n + SCAN_CHUNK - 1) / SCAN_CHUNK : 1;
    launch_begin(p, "scan_reduce", s);
    k_scan_reduce<<<nb, SCAN_THREADS, 0, s>>>(in, n, p->scan_sums);
    launch_end(p, s);
    launch_begin(p, "scan_apply", s);
    k_scan_apply<<<nb, SCAN_THREADS, 0, s>>>(in, out, n, p->scan_sums);
    launch_end(p, s);
    return cudaGetLastError();
}

cudaError_t phase_table_init() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    std::vector<double2> t(2 * PHASE_TAB_HALF + 1);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int k = -PHASE_TAB_HALF; k <= PHASE_TAB_HALF; ++k) {
        const long double a = pi * (long double)k / (long double)PHASE_TAB_HALF;
        t[k + PHASE_TAB_HALF] = make_double2((double)sinl(a), (double)cosl(a));
    }
    // exact values where the angle is a multiple of pi/2
    for (int k : {-PHASE_TAB_HALF, -PHASE_TAB_HALF / 2, 0, PHASE_TAB_HALF / 2, PHASE_TAB_HALF}) {
        const int q = ((k / (PHASE_TAB_HALF / 2)) % 4 + 4) % 4;
        t[k + PHASE_TAB_HALF] = make_double2(q == 1 ? 1.0 : (q == 3 ? -1.0 : 0.0), q == 0 ? 1.0 : (q == 2 ? -1.0 : 0.0));
    }
    e = cudaMemcpyToSymbol(g_phase_tab, t.data(), t.size() * sizeof(double2));
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

cudaError_t run_pattern(Plan* p, cudaStream_t s) {
    const int N = (int)p->N, Ms = (int)p->Ms, nkeys = 2 * Ms;
    cudaError_t e = cudaMemsetAsync(p->counters, 0, CNT_N * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->bucket, 0, (size_t)(nkeys + 1) * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->cursor, 0, (size_t)nkeys * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;

    launch_begin(p, "bucket_count", s);
    k_bucket_count<<<blocks_for(N, 256), 256, 0, s>>>(p->x, N, Ms, p->bucket, p->counters);
    launch_end(p, s);
    if ((e = run_exclusive_scan(p, p->bucket, p->bucket, nkeys, s)) != cudaSuccess) return e;
    launch_begin(p, "bucket_scatter", s);
    k_bucket_scatter<<<blocks_for(N, 256), 256, 0, s>>>(p->x, N, Ms, p->bucket, p->cursor, p->perm, p->skey);
    launch_end(p, s);
    launch_begin(p, "bucket_fixup", s);
    k_bucket_fixup<<<blocks_for(nkeys, 256), 256, 0, s>>>(p->bucket, nkeys, p->perm, p->seg_list, p->counters);
    launch_end(p, s);
    launch_begin(p, "bigseg_fixup", s);
    k_bigseg_fixup<<<p->sms, 256, 0, s>>>(p->seg_list, p->counters, p->bucket, p->perm, p->sort_tmp);
    launch_end(p, s);
    launch_begin(p, "gather_nodes", s);
    k_gather_nodes<<<blocks_for(N, 256), 256, 0, s>>>(p->x, p->perm, N, (double)p->M, p->xs, p->phase);
    launch_end(p, s);

    launch_begin(p, "col_ranges", s);
    k_col_ranges<<<blocks_for(Ms, 256), 256, 0, s>>>(p->bucket, N, Ms, p->m, p->col_start, p->col_count,
                                                     p->counters);
    launch_end(p, s);
    return run_exclusive_scan(p, p->col_count, p->col_off, Ms, s);
}

// ---- the pattern of every problem of a batch in one launch ----------------------------
//
// One CTA per problem (persistent CTAs take problems in the order given, largest first): the
// same steps as run_pattern -- clear, key histogram, its exclusive scan (the bucket offsets),
// scatter, ordering of each bucket by caller index, sorted nodes and phases, column ranges and
// their scan -- separated by CTA barriers instead of kernel boundaries.  The results are those
// of run_pattern on each problem.

namespace {

constexpr int BP_THREADS = 1024;

// out[i] = sum_{q < i} in[q] for i < n and out[n] = the total (out may alias in); every thread
// of the CTA calls it.  Thread t scans the contiguous range [t per, (t + 1) per).
INFFT_D void cta_exclusive_scan(const int32_t* in, int32_t* out, int n, int32_t* red) {
    const int per = (n + BP_THREADS - 1) / BP_THREADS;
    const int a = min((int)threadIdx.x * per, n), b = min(a + per, n);
    int32_t loc = 0;
    for (int i = a; i < b; ++i) loc += in[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t inc = loc;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) red[w] = inc;
    __syncthreads();
    int32_t run = inc - loc;
    for (int ww = 0; ww < w; ++ww) run += red[ww];
    for (int i = a; i < b; ++i) {
        const int32_t v = in[i];
        out[i] = run;
        run += v;
    }
    if (threadIdx.x == BP_THREADS - 1) out[n] = run;
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(BP_THREADS)
k_batch_pattern(const PatternArgs* __restrict__ probs, const int32_t* __restrict__ order, int P) {
    __shared__ int32_t red[BP_THREADS / 32];
    const int tid = threadIdx.x;
    for (int k = blockIdx.x; k < P; k += gridDim.x) {
        const PatternArgs a = probs[order[k]];
        const int N = a.N, Ms = a.Ms, nkeys = 2 * Ms;
        // clear
        for (int i = tid; i <= nkeys; i += BP_THREADS) a.bucket[i] = 0;
        for (int i = tid; i < nkeys; i += BP_THREADS) a.cursor[i] = 0;
        if (tid < CNT_N) a.counters[tid] = 0;
        __syncthreads();
        // key histogram (bad nodes counted, and keyed as x = 0)
        for (int j = tid; j < N; j += BP_THREADS) {
            const double xj = a.x[j];
            if (!(isfinite(xj) && xj >= -0.5 && xj < 0.5)) atomicAdd(&a.counters[CNT_BAD_NODES], 1);
            atomicAdd(&a.bucket[node_key(checked_node(a.x, j), Ms)], 1);
        }
        __syncthreads();
        cta_exclusive_scan(a.bucket, a.bucket, nkeys, red);
        // scatter
        for (int j = tid; j < N; j += BP_THREADS) {
            const uint32_t key = node_key(checked_node(a.x, j), Ms);
            const int pos = a.bucket[key] + atomicAdd(&a.cursor[key], 1);
            a.perm[pos] = j;
            a.skey[pos] = key;
        }
        __syncthreads();
        // order each bucket by caller index: small ones by one thread, large ones by the CTA
        for (int b = tid; b < nkeys; b += BP_THREADS) {
            const int s0 = a.bucket[b], s1 = a.bucket[b + 1], c = s1 - s0;
            if (c <= 1) continue;
            if (c > SMALL_BUCKET) {
                a.seg_list[atomicAdd(&a.counters[CNT_BIG_SEGMENTS], 1)] = b;
                continue;
            }
            for (int i = s0 + 1; i < s1; ++i) {
                const int v = a.perm[i];
                int q = i - 1;
                while (q >= s0 && a.perm[q] > v) {
                    a.perm[q + 1] = a.perm[q];
                    --q;
                }
                a.perm[q + 1] = v;
            }
        }
        __syncthreads();
        const int nbig = a.counters[CNT_BIG_SEGMENTS];
        for (int it = 0; it < nbig; ++it) {
            const int b = a.seg_list[it];
            const int s0 = a.bucket[b], c = a.bucket[b + 1] - s0;
            for (int i = tid; i < c; i += BP_THREADS) {
                const int v = a.perm[s0 + i];
                int rank = 0;
                for (int q = 0; q < c; ++q) rank += a.perm[s0 + q] < v;
                a.sort_tmp[s0 + rank] = v;
            }
            __syncthreads();
            for (int i = tid; i < c; i += BP_THREADS) a.perm[s0 + i] = a.sort_tmp[s0 + i];
            __syncthreads();
        }
        // sorted nodes and their phases
        for (int i = tid; i < N; i += BP_THREADS) {
            const double xi = checked_node(a.x, a.perm[i]);
            a.xs[i] = xi;
            a.phase[i] = node_phase(a.M, xi);
        }
        // column ranges: keys [2(p-m), 2(p+m)] (mod 2 M_sigma)
        for (int p = tid; p < Ms; p += BP_THREADS) {
            int lo = p - a.m; if (lo < 0) lo += Ms;
            int hi = p + a.m; if (hi >= Ms) hi -= Ms;
            const int klo = 2 * lo, khi = 2 * hi + 1;
            const int s0 = a.bucket[klo], s1 = a.bucket[khi];
            const int c = (klo < khi) ? (s1 - s0) : (N - s0) + s1;
            a.col_start[p] = (s0 == N) ? 0 : s0;
            a.col_count[p] = c;
            if (c == 0) atomicAdd(&a.counters[CNT_EMPTY], 1);
            atomicMax(&a.counters[CNT_MAX_COLUMN], c);
        }
        __syncthreads();
        cta_exclusive_scan(a.col_count, a.col_off, Ms, red);
    }
}

cudaError_t run_pattern_batch(const PatternArgs* probs, const int32_t* order, int P, int sms, cudaStream_t s) {
    const int ctas = std::min(P, 2 * sms);
    k_batch_pattern<<<ctas, BP_THREADS, 0, s>>>(probs, order, P);
    count_launches(1);
    return cudaGetLastError();
}
