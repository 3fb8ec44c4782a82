// Two-dimensional tensor-product form of the modified adjoint NFFT: the method of
// Sec. 3.2.2 taken per dimension (the paper treats d = 1; Sec. 5 leaves d > 1 open).
//
//   pattern : nodes are counting-sorted by grid cell (c1, c2), c_t = floor(M_sigma,t x_t)
//             + M_sigma,t/2, and ordered by node index inside a cell.  The candidates of
//             column l are the nodes of the (2m+1)^2 cells around it; a candidate enters
//             I(l) by the exact test of eq:set_xj in each dimension, decided on
//             u_t = fl(M_sigma,t x_t).  One warp per column: a counting pass, a scan and a
//             filling pass whose ballot ranks keep the candidate order (deterministic).
//   B_opt   : per column the fp64 normal equations (Re G_l + mu I) b = Re r_l of
//             eq:opt_ansatz2 .. eq:solution_ansatz2 (real b, Tikhonov mu = tau Re kappa(0)),
//             Gram entries Re[kappa_1(d_1) kappa_2(d_2)] of the product kernel.
//             Columns of up to 128 nodes: one CTA each, one thread per row, packed
//             triangle in shared memory, right-looking Cholesky with the forward solve
//             fused.  Larger columns: one CTA each, largest first, packed triangle in a
//             global scratch slot, Cholesky blocked by PB columns: the PB x PB diagonal
//             block in shared memory, the rows below by a row-wise triangular solve, the
//             trailing update in TB x TB tiles whose panel slices are staged in shared
//             memory (4 x 4 register blocks per thread).
//   apply   : one warp per column gathers g_l = sum_j b_lj f_j (fp32; fp64 weights and
//             accumulation for columns with ||b_l||_1 > 32), then the 2-D FFT: rows
//             (length M_sigma,2, the kept k2 stored transposed) and the kept columns
//             (length M_sigma,1), with (-1)^(k1+k2) d_k fused into the last store.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "plan.h"
#include "fft_device.cuh"

struct infft2d_plan_s {
    int device = 0;
    int64_t M1 = 0, M2 = 0, Ms1 = 0, Ms2 = 0, N = 0, P = 0;
    int m = 0, kernel = INFFT_KERNEL_FULL, log1 = 0, log2 = 0;
    double sigma = 2.0, tau = 1e-12;
    int64_t nnz_cap = 0, nnz = 0;
    int max_column = 0;

    double2* x = nullptr;          // N nodes, caller order
    double2* xs = nullptr;         // N nodes, sorted by cell
    int32_t* node_cell = nullptr;  // N: cell of each node (-1: invalid node)
    int32_t* perm = nullptr;       // N: sorted position -> caller index
    int32_t* cell_start = nullptr; // P + 1: node counts per cell, then their exclusive prefix
    int32_t* cursor = nullptr;     // P: scatter cursors
    int32_t* big_cells = nullptr;  // P: cells with more than 32 nodes (ordered by one CTA each)
    int32_t* col_off = nullptr;    // P + 1
    int32_t* col_node = nullptr;   // nnz_cap: caller index of each entry, column by column
    int32_t* lists = nullptr;      // 5 P: columns of the three shared-memory tiers and the two large tiers
    int32_t* order = nullptr;      // P: large columns, largest first
    int32_t* spread_big = nullptr; // P: columns above SPREAD_BIG entries
    int spread_big_count = 0;
    int32_t* hist = nullptr;       // LARGE_NMAX + 2: size buckets, then offsets / cursors; ticket
    int32_t* counters = nullptr;   // C2_N
    float* w32 = nullptr;          // nnz_cap
    uint8_t* kind = nullptr;       // P: column kinds of the fp32 spread (K2_WIDE, K2_INDEXED)
    float2* fsort = nullptr;       // N: the data in sorted node order (fp32 spread of run columns)
    float* wlo = nullptr;          // nnz_cap: fp32(b - fp32(b)), the low part of wide columns' weights
    double* w64 = nullptr;         // nnz_cap
    double* J = nullptr;           // P
    uint8_t* wide = nullptr;       // P
    void* grid = nullptr;          // P complex128 (also used as complex64)
    void* work = nullptr;          // M2 Ms1 complex128: the row transforms, transposed
    void* stage_in = nullptr;      // max(N, M1 M2) complex128
    void* stage_out = nullptr;
    void* arena = nullptr;
    double* scratch = nullptr;     // large-column triangles (owned, grown on demand)
    size_t scratch_doubles = 0;
    double* gscratch = nullptr;    // triangles of the columns factored by many CTAs (owned)
    size_t gscratch_doubles = 0;
    void* gdesc = nullptr;         // their descriptors (owned)
    int gdesc_cap = 0;
    int32_t* gprefix = nullptr;    // per panel step, the exclusive tile prefix over those columns (owned)
    size_t gprefix_cap = 0;
    int nodes_set = 0, precomputed = 0;
    cudaStream_t last_stream = nullptr;
};

namespace {

enum {
    C2_BAD = 0, C2_FALLBACK = 1, C2_UNSUPPORTED = 2, C2_MAX_COLUMN = 3, C2_EMPTY = 4,
    C2_LIST0 = 5,   // C2_LIST0 + t: length of the list of tier t (0..2 shared memory, 3 one CTA, 4 many CTAs)
    C2_BIG_CELLS = 10, C2_WIDE = 11,
    C2_SPREAD_BIG = 12,   // columns above SPREAD_BIG entries, spread by a whole CTA each
    C2_INDEXED = 13,      // columns the fp32 spread reads through node indices
    C2_N = 14
};

constexpr int TIER_NMAX[3] = {32, 64, 128};
constexpr int LARGE_NMAX = 8192;
constexpr int GIANT_N = 384;      // columns above this are factored by many CTAs
constexpr size_t GIANT_BUDGET = (size_t)16 << 30;   // bytes of giant triangles factored at once
constexpr int PB = 16;             // panel width of the blocked solver
constexpr int TB = 64;             // trailing-update tile
constexpr int TBP = TB + 2;        // shared-memory row stride of the staged panel slices
constexpr int LARGE_THREADS = 256;
constexpr int CELL_SORT_MAX = 4096;
constexpr int FFT2_THREADS = 256;
constexpr int SPREAD_LPC = 4;     // lanes per column of the fp32 spread (each takes every fourth cell-row run)
constexpr int SPREAD_BIG = 512;   // longer columns are spread by one CTA each

thread_local std::string g_err2;

infft_status fail2(infft_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(st, "%s", buf);
}

infft_status cuda_fail2(cudaError_t e, const char* what) {
    return fail2(e == cudaErrorMemoryAllocation ? INFFT_ENOMEM : INFFT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct DeviceGuard2 {
    int prev = -1;
    explicit DeviceGuard2(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard2() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool on_device2(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---- kernel entries (Gram and right-hand side) -------------------------------

struct K2 {
    double M1, M2;   // band sizes
    double K1, K2;   // Dirichlet frequencies per dimension: M (full) or M - 1 (sym)
    double inv;      // 1 / (M_sigma,1 M_sigma,2)
    double diag;     // Re kappa(0)
    int sym;
    int shortd;      // every kernel argument pi d is at most 0.25: sin(pi d), cos(pi (d1 + d2)) by series
};

// a - b as the representative in [-1/2, 1/2] on the torus; across the seam the
// +-1/2 shifts go to the operands first, so close nodes keep their difference exactly
INFFT_D double tdiff(double a, double b) {
    double d = a - b;
    if (d > 0.5) d = (a - 0.5) - (b + 0.5);
    else if (d < -0.5) d = (a + 0.5) - (b - 0.5);
    return d;
}

constexpr double PI_D = 3.141592653589793;

// Taylor series of sin x and cos x (|x| <= 0.5 where used; the first omitted terms,
// x^17/17! and x^18/18!, stay below 1e-20 relative)
INFFT_D double sin_series(double x) {
    const double x2 = x * x;
    double q = 1.0;
#pragma unroll
    for (int k = 14; k >= 2; k -= 2) q = fma(-x2 * (1.0 / (double)(k * (k + 1))), q, 1.0);   // folded constants
    return x * q;
}
INFFT_D double cos_series(double x) {
    const double x2 = x * x;
    double q = 1.0;
#pragma unroll
    for (int k = 15; k >= 1; k -= 2) q = fma(-x2 * (1.0 / (double)(k * (k + 1))), q, 1.0);
    return q;
}

// A point of the kernel's argument: its coordinates and, per dimension, (sin, cos)(pi K_t x_t)
struct NodeK {
    double x1, x2, s1, c1, s2, c2;
};

// (sin, cos)(pi K x) with K x split exactly (K x = h + lo by an FMA), h reduced modulo 2
// exactly, and the tiny lo added to first order
INFFT_D void phase_pi(double K, double x, double& s, double& c) {
    const double h = K * x;
    const double lo = fma(K, x, -h);
    const double hr = h - 2.0 * rint(0.5 * h);
    double sn, cs;
    sincospi(hr, &sn, &cs);
    const double e = PI_D * lo;
    s = fma(e, cs, sn);
    c = fma(-e, sn, cs);
}

INFFT_D NodeK node_k(double2 x, const K2& k) {
    NodeK n;
    n.x1 = x.x;
    n.x2 = x.y;
    phase_pi(k.K1, x.x, n.s1, n.c1);
    phase_pi(k.K2, x.y, n.s2, n.c2);
    return n;
}

// sin(pi K d) and sin(pi d) for the torus difference d = a - b (at d = 0: K and 1, the
// ratio's limit).  sin(pi K d) comes from the two points' phases, sin(pi K (a - b)) =
// s_a c_b - c_a s_b, which changes sign with d -> d -+ 1 when K is odd; where |K d| < 1/8
// that difference would lose relative accuracy and sinpi(K d) is evaluated instead.
INFFT_D void dirichlet_parts(double a, double sa, double ca, double b, double sb, double cb, double K, bool oddK,
                             bool shortd, double& num, double& den, double& d) {
    d = tdiff(a, b);
    if (d == 0.0) { num = K; den = 1.0; return; }
    const double kd = K * d;
    if (fabs(kd) < 0.125) {
        num = sinpi(kd);
    } else {
        num = sa * cb - ca * sb;
        if (oddK && fabs(a - b) > 0.5) num = -num;
    }
    den = shortd ? sin_series(PI_D * d) : sinpi(d);
}

// Re kappa(a - b) = Re[kappa_1(d_1) kappa_2(d_2)]: full kernel kappa_t(d) = e^{-i pi d} sin(pi M d)/
// (M_sigma sin(pi d)), so the real part carries cos(pi (d_1 + d_2)); sym kernel: real Dirichlet
// kernels sin(pi (M - 1) d)/(M_sigma sin(pi d)) (Remark remark:Dirichlet_ansatz2 per dimension)
INFFT_D double re_kappa2(const NodeK& a, const NodeK& b, const K2& k) {
    double n1, e1, d1, n2, e2, d2;
    dirichlet_parts(a.x1, a.s1, a.c1, b.x1, b.s1, b.c1, k.K1, k.sym, k.shortd, n1, e1, d1);
    dirichlet_parts(a.x2, a.s2, a.c2, b.x2, b.s2, b.c2, k.K2, k.sym, k.shortd, n2, e2, d2);
    double v = (n1 * n2) / (e1 * e2) * k.inv;
    if (!k.sym) v *= k.shortd ? cos_series(PI_D * (d1 + d2)) : cospi(d1 + d2);
    return v;
}

// the grid point of column p as a kernel argument (l_t / M_sigma,t is exact)
INFFT_D NodeK column_point(int p, int Ms1, int Ms2, const K2& k) {
    return node_k(make_double2((double)(p / Ms2 - Ms1 / 2) / (double)Ms1, (double)(p % Ms2 - Ms2 / 2) / (double)Ms2),
                  k);
}

INFFT_D int trow(int i) { return i * (i + 1) / 2; }

// ---- pattern ------------------------------------------------------------------

__global__ void k2_cells(const double2* __restrict__ x, int N, int Ms1, int Ms2, int32_t* __restrict__ node_cell,
                         int32_t* __restrict__ cell_count, int32_t* __restrict__ counters) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double2 v = x[j];
    if (!(v.x >= -0.5 && v.x < 0.5 && v.y >= -0.5 && v.y < 0.5)) {   // NaN fails too
        node_cell[j] = -1;
        atomicAdd(&counters[C2_BAD], 1);
        return;
    }
    const int c1 = (int)floor((double)Ms1 * v.x) + Ms1 / 2;
    const int c2 = (int)floor((double)Ms2 * v.y) + Ms2 / 2;
    const int c = c1 * Ms2 + c2;
    node_cell[j] = c;
    atomicAdd(&cell_count[c], 1);
}

// exclusive prefix of a[0 .. n) in place, total in a[n] (one CTA of 1024 threads)
__global__ void __launch_bounds__(1024) k2_scan(int32_t* __restrict__ a, int n) {
    __shared__ int32_t part[1024];
    const int per = (n + 1023) / 1024;
    const int lo = min(threadIdx.x * per, n), hi = min(lo + per, n);
    int32_t s = 0;
    for (int i = lo; i < hi; ++i) s += a[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const int32_t v = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int i = lo; i < hi; ++i) {
        const int32_t c = a[i];
        a[i] = run;
        run += c;
    }
    if (threadIdx.x == 1023) a[n] = part[1023];
}

__global__ void k2_scatter(const int32_t* __restrict__ node_cell, int N, const int32_t* __restrict__ cell_start,
                           int32_t* __restrict__ cursor, int32_t* __restrict__ perm) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int c = node_cell[j];
    if (c < 0) return;
    perm[cell_start[c] + atomicAdd(&cursor[c], 1)] = j;
}

// order the nodes of each cell by caller index: cells of up to 32 nodes by one thread,
// larger ones are listed for k2_cell_sort_big
__global__ void k2_cell_sort(const int32_t* __restrict__ cell_start, int P, int32_t* __restrict__ perm,
                             int32_t* __restrict__ big_cells, int32_t* __restrict__ counters) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P) return;
    const int s = cell_start[c], n = cell_start[c + 1] - s;
    if (n <= 1) return;
    if (n > 32) {
        big_cells[atomicAdd(&counters[C2_BIG_CELLS], 1)] = c;
        return;
    }
    for (int i = 1; i < n; ++i) {
        const int v = perm[s + i];
        int k = i - 1;
        while (k >= 0 && perm[s + k] > v) {
            perm[s + k + 1] = perm[s + k];
            --k;
        }
        perm[s + k + 1] = v;
    }
}

// one CTA per listed cell: rank sort of its (distinct) caller indices; cells above
// CELL_SORT_MAX nodes keep the scatter order (valid, not reproducible run to run)
__global__ void __launch_bounds__(256) k2_cell_sort_big(const int32_t* __restrict__ cell_start,
                                                        int32_t* __restrict__ perm,
                                                        const int32_t* __restrict__ big_cells,
                                                        const int32_t* __restrict__ counters) {
    __shared__ int32_t v[CELL_SORT_MAX];
    const int cnt = counters[C2_BIG_CELLS];
    for (int b = blockIdx.x; b < cnt; b += gridDim.x) {
        const int c = big_cells[b];
        const int s = cell_start[c], n = cell_start[c + 1] - s;
        if (n > CELL_SORT_MAX) continue;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = perm[s + i];
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int vi = v[i];
            int r = 0;
            for (int k = 0; k < n; ++k) r += v[k] < vi;
            perm[s + r] = vi;
        }
    }
}

__global__ void k2_gather_nodes(const double2* __restrict__ x, const int32_t* __restrict__ perm,
                                const int32_t* __restrict__ cell_start, int P, double2* __restrict__ xs) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cell_start[P]) return;
    xs[q] = x[perm[q]];
}

// does the node coordinate xt put grid index a (= l + M_sigma/2) into its set (eq:set_xj)?
// l in [ceil(u) - m, floor(u) + m] mod M_sigma, u = fl(M_sigma xt); with c = floor(u) + M_sigma/2,
// a - c lies in [1 - m, m] (mod M_sigma), or equals -m when u is an integer
INFFT_D bool covers(int a, double xt, int Ms, int m) {
    const double u = (double)Ms * xt;
    const double fu = floor(u);
    const int c = (int)fu + Ms / 2;
    int d = (a - c + m) % Ms;
    if (d < 0) d += Ms;
    d -= m;
    return d <= m && (d > -m || u == fu);
}

// One warp per column p = a1 Ms2 + a2: candidates in the cells (a1 + d1, a2 - m .. a2 + m)
// for d1 = -m .. m (wrapped; the c2 range is at most two runs of consecutive cells)
template <bool FILL>
__global__ void __launch_bounds__(256) k2_columns(const double2* __restrict__ xs, const int32_t* __restrict__ perm,
                                                  const int32_t* __restrict__ cell_start, int Ms1, int Ms2, int m,
                                                  int32_t* __restrict__ col_count, const int32_t* __restrict__ col_off,
                                                  int32_t* __restrict__ col_node, int32_t* __restrict__ counters) {
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (p >= Ms1 * Ms2) return;
    const int a1 = p / Ms2, a2 = p - a1 * Ms2;
    const int out = FILL ? col_off[p] : 0;
    const unsigned below = lanemask_lt();
    int cnt = 0;
    int r0[2], r1[2], nr = 1;
    const int lo = a2 - m, hi = a2 + m;
    if (lo < 0) { r0[0] = lo + Ms2; r1[0] = Ms2 - 1; r0[1] = 0; r1[1] = hi; nr = 2; }
    else if (hi >= Ms2) { r0[0] = lo; r1[0] = Ms2 - 1; r0[1] = 0; r1[1] = hi - Ms2; nr = 2; }
    else { r0[0] = lo; r1[0] = hi; }
    for (int d1 = -m; d1 <= m; ++d1) {
        const int c1 = (a1 + d1 + Ms1) % Ms1;
        for (int r = 0; r < nr; ++r) {
            const int s = cell_start[c1 * Ms2 + r0[r]], e = cell_start[c1 * Ms2 + r1[r] + 1];
            for (int base = s; base < e; base += 32) {
                const int q = base + lane;
                bool in = false;
                if (q < e) {
                    const double2 v = xs[q];
                    in = covers(a1, v.x, Ms1, m) && covers(a2, v.y, Ms2, m);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                if (FILL && in) col_node[out + cnt + __popc(bal & below)] = perm[q];
                cnt += __popc(bal);
            }
        }
    }
    if (!FILL && lane == 0) {
        col_count[p] = cnt;
        atomicMax(&counters[C2_MAX_COLUMN], cnt);
        if (cnt == 0) atomicAdd(&counters[C2_EMPTY], 1);
    }
}

// ---- precompute: routing ------------------------------------------------------

__global__ void k2_route(const int32_t* __restrict__ col_off, int P, int32_t* __restrict__ lists,
                         double* __restrict__ w64, float* __restrict__ w32, double* __restrict__ J,
                         uint8_t* __restrict__ wide, int32_t* __restrict__ hist, int32_t* __restrict__ spread_big,
                         int32_t* __restrict__ counters) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int off = col_off[p], n = col_off[p + 1] - off;
    wide[p] = 0;
    if (n > SPREAD_BIG) spread_big[atomicAdd(&counters[C2_SPREAD_BIG], 1)] = p;
    if (n == 0) { J[p] = 1.0; return; }
    if (n > LARGE_NMAX) {   // not built: b_l = 0 (J_l = 1)
        for (int i = 0; i < n; ++i) { w64[off + i] = 0.0; w32[off + i] = 0.0f; }
        J[p] = 1.0;
        atomicAdd(&counters[C2_UNSUPPORTED], 1);
        return;
    }
    const int t = n <= TIER_NMAX[0] ? 0 : n <= TIER_NMAX[1] ? 1 : n <= TIER_NMAX[2] ? 2 : n <= GIANT_N ? 3 : 4;
    lists[t * P + atomicAdd(&counters[C2_LIST0 + t], 1)] = p;
    if (t == 3) atomicAdd(&hist[LARGE_NMAX - n], 1);
}

// the large list in largest-first order (counting sort by size, descending)
__global__ void k2_order_large(const int32_t* __restrict__ col_off, const int32_t* __restrict__ large, int P,
                               int32_t* __restrict__ cursor, int32_t* __restrict__ order,
                               const int32_t* __restrict__ counters) {
    const int cnt = counters[C2_LIST0 + 3];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int p = large[i];
        const int n = col_off[p + 1] - col_off[p];
        order[atomicAdd(&cursor[LARGE_NMAX - n], 1)] = p;
    }
}

// ---- precompute: columns of up to NMAX nodes (one CTA of NMAX threads each) ---

template <int NMAX> constexpr size_t small_smem() {
    return (size_t)(NMAX * (NMAX + 1) / 2 + 3 * NMAX) * sizeof(double) + NMAX * sizeof(NodeK);
}

template <int NMAX>
__global__ void __launch_bounds__(NMAX) k2_solve_small(const double2* __restrict__ x, const int32_t* __restrict__ col_off,
                                                       const int32_t* __restrict__ col_node,
                                                       const int32_t* __restrict__ list, int list_id, int Ms1,
                                                       int Ms2, K2 kp, double mu0, double* __restrict__ w64,
                                                       float* __restrict__ w32, double* __restrict__ J,
                                                       uint8_t* __restrict__ wide, int32_t* __restrict__ counters) {
    extern __shared__ __align__(16) double sm2[];
    double* A = sm2;                                   // packed lower triangle, row-major
    double* r = A + NMAX * (NMAX + 1) / 2;             // right-hand side, then y
    double* lk = r + NMAX;                             // two buffers of L's current column
    NodeK* xl = (NodeK*)(lk + 2 * NMAX);               // the column's nodes with their phases
    __shared__ double red[2 * (NMAX / 32 > 0 ? NMAX / 32 : 1)];
    const int i = threadIdx.x;                         // this thread's row
    const int count = counters[C2_LIST0 + list_id];
    for (int it = blockIdx.x; it < count; it += gridDim.x) {
        const int p = list[it];
        const int off = col_off[p], n = col_off[p + 1] - off;
        const NodeK cp = column_point(p, Ms1, Ms2, kp);
        __syncthreads();
        if (i < n) xl[i] = node_k(x[col_node[off + i]], kp);
        __syncthreads();
        double mu = mu0, ysq = 0.0;
        bool ok = false;
        for (int attempt = 0; attempt < 3 && !ok; ++attempt) {
            // the packed triangle's entries are spread evenly over the CTA's threads (a thread
            // per row would leave the short rows' threads idle); row of entry e by an fp32 square
            // root, corrected exactly
            const int ntri = n * (n + 1) / 2;
            for (int e = i; e < ntri; e += NMAX) {
                int a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
                while (trow(a + 1) <= e) ++a;
                while (trow(a) > e) --a;
                const int c = e - trow(a);
                A[e] = (a == c) ? kp.diag + mu : re_kappa2(xl[a], xl[c], kp);
            }
            if (i < n) r[i] = re_kappa2(cp, xl[i], kp);
            __syncthreads();
            ysq = 0.0;
            bool failed = false;
            for (int k = 0; k < n; ++k) {
                const double akk = A[trow(k) + k];
                if (!(akk > 0.0) || !isfinite(akk)) { failed = true; break; }   // CTA-uniform
                const double rp = rsqrt(akk);
                const double yk = r[k] * rp;
                ysq = fma(yk, yk, ysq);
                double* l = lk + (k & 1) * NMAX;
                if (i > k && i < n) l[i] = A[trow(i) + k] * rp;
                __syncthreads();
                if (i > k && i < n) {
                    const double li = l[i];
                    A[trow(i) + k] = li;
                    for (int j = k + 1; j <= i; ++j) A[trow(i) + j] = fma(-li, l[j], A[trow(i) + j]);
                    r[i] = fma(-li, yk, r[i]);
                }
                if (i == k) { A[trow(k) + k] = rp; r[k] = yk; }
                __syncthreads();
            }
            ok = !failed;
            if (!ok) mu *= 1e3;
            __syncthreads();
        }
        if (!ok) {
            if (i < n) { w64[off + i] = 0.0; w32[off + i] = 0.0f; }
            if (i == 0) { J[p] = 1.0; atomicAdd(&counters[C2_FALLBACK], 1); }
            continue;
        }
        if (i == 0 && mu != mu0) atomicAdd(&counters[C2_FALLBACK], 1);
        // back solve L^T b = y: b_k = y_k rp_k after rows k' > k were taken out;
        // then row k of L removes b_k from the remaining entries
        double bsq = 0.0, babs = 0.0;
        for (int k = n - 1; k >= 0; --k) {
            const double bk = r[k] * A[trow(k) + k];
            if (i < k) r[i] = fma(-A[trow(k) + i], bk, r[i]);
            if (i == k) {
                w64[off + k] = bk;
                w32[off + k] = (float)bk;
                bsq = bk * bk;
                babs = fabs(bk);
            }
            __syncthreads();
        }
        for (int o = 16; o; o >>= 1) {
            bsq += __shfl_xor_sync(0xffffffffu, bsq, o);
            babs += __shfl_xor_sync(0xffffffffu, babs, o);
        }
        constexpr int W = NMAX / 32 > 0 ? NMAX / 32 : 1;
        if ((i & 31) == 0) { red[i >> 5] = bsq; red[W + (i >> 5)] = babs; }
        __syncthreads();
        if (i == 0) {
            double t = 0.0, a = 0.0;
            for (int w = 0; w < W; ++w) { t += red[w]; a += red[W + w]; }
            J[p] = 1.0 - ysq - mu * t;
            const bool wd = a > WIDE_COLUMN_L1;
            wide[p] = wd;
            if (wd) atomicAdd(&counters[C2_WIDE], 1);
        }
    }
}

// ---- precompute: large columns (blocked, triangle in global memory) -------------
//
// Building blocks shared by the one-CTA-per-column solver (columns of 129 .. GIANT_N
// nodes) and the multi-CTA solver of the largest columns.  A is a packed lower
// triangle (row i at i(i+1)/2, the diagonal holding the reciprocal pivot once
// factored); r is the right-hand side, overwritten by y and then by the back solve.

struct PanelShared {
    double D[PB * (PB + 1)];   // diagonal block
    double ypan[PB];           // y of the block's columns
    double ysq;                // running |y|^2
    int fail;
};

// One panel step at column kb (whole CTA, ends with __syncthreads): the PB x PB diagonal
// block is factored by warp 0 in shared memory together with its part of y = L^{-1} r; the
// rows below are solved row by row (L_ib = (A_ib - sum_{b'<b} L_ib' L_bb') / L_bb) and
// take y out of r.  A failed pivot sets ps.fail (CTA-uniform after the return).
INFFT_D void panel_step(double* __restrict__ A, double* __restrict__ r, int n, int kb, PanelShared& ps) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int w = min(PB, n - kb);
    double* D = ps.D;
    double* ypan = ps.ypan;
    for (int e = tid; e < PB * PB; e += blockDim.x) {
        const int a = e / PB, b = e % PB;
        D[a * (PB + 1) + b] = (a < w && b <= a) ? A[trow(kb + a) + kb + b] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
        bool bad = false;
        for (int c = 0; c < w; ++c) {
            const double akk = D[c * (PB + 1) + c];
            if (!(akk > 0.0) || !isfinite(akk)) { bad = true; break; }   // warp-uniform
            const double rp = rsqrt(akk);
            __syncwarp();
            if (lane > c && lane < w) D[lane * (PB + 1) + c] *= rp;
            __syncwarp();
            if (lane > c && lane < w) {
                const double li = D[lane * (PB + 1) + c];
                for (int b = c + 1; b <= lane; ++b)
                    D[lane * (PB + 1) + b] = fma(-li, D[b * (PB + 1) + c], D[lane * (PB + 1) + b]);
            }
            __syncwarp();
            if (lane == 0) D[c * (PB + 1) + c] = rp;
            __syncwarp();
        }
        if (lane == 0) {
            if (bad) {
                ps.fail = 1;
            } else {
                double ysq = ps.ysq;
                for (int c = 0; c < w; ++c) {
                    double v = r[kb + c];
                    for (int b = 0; b < c; ++b) v = fma(-D[c * (PB + 1) + b], ypan[b], v);
                    v *= D[c * (PB + 1) + c];
                    ypan[c] = v;
                    r[kb + c] = v;
                    ysq = fma(v, v, ysq);
                }
                ps.ysq = ysq;
            }
        }
    }
    __syncthreads();
    if (ps.fail) return;
    for (int e = tid; e < PB * PB; e += blockDim.x) {
        const int a = e / PB, b = e % PB;
        if (a < w && b <= a) A[trow(kb + a) + kb + b] = D[a * (PB + 1) + b];
    }
    // the diagonal block is read through a volatile view: loaded at each use from shared
    // memory (a broadcast) rather than held in 136 registers across the row loop
    const volatile double* Dv = D;
    for (int i = kb + w + tid; i < n; i += blockDim.x) {
        double v[PB];
        double* row = A + trow(i) + kb;
#pragma unroll
        for (int b = 0; b < PB; ++b) v[b] = b < w ? row[b] : 0.0;
        double acc = r[i];
#pragma unroll
        for (int b = 0; b < PB; ++b) {
            if (b < w) {
                double s = v[b];
#pragma unroll
                for (int c = 0; c < b; ++c) s = fma(-v[c], Dv[b * (PB + 1) + c], s);
                v[b] = s * Dv[b * (PB + 1) + b];
                acc = fma(-v[b], ypan[b], acc);
            }
        }
#pragma unroll
        for (int b = 0; b < PB; ++b)
            if (b < w) row[b] = v[b];
        r[i] = acc;
    }
    __syncthreads();
}

// number of TB x TB lower-triangular tiles of the trailing matrix after the panel at kb
INFFT_HD int trailing_tiles(int n, int kb) {
    const int T = n - kb - PB;
    if (T <= 0) return 0;
    const int nt = (T + TB - 1) / TB;
    return nt * (nt + 1) / 2;
}

// tile index -> (ti, tj), tj <= ti, row-major over the lower triangle of tiles
INFFT_D void tile_coords(int tile, int& ti, int& tj) {
    ti = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);
    while (trow(ti + 1) <= tile) ++ti;
    while (trow(ti) > tile) --ti;
    tj = tile - trow(ti);
}

// A_ij -= sum_c L_ic L_jc over the panel columns kb .. kb + PB - 1, for the tile (ti, tj) of
// the rows / columns from kb + PB (whole CTA of 256 threads, 4 x 4 entries each; the panel
// slices of the tile's rows and columns are staged in Li, Lj with row stride TBP)
INFFT_D void trailing_tile(double* __restrict__ A, int n, int kb, int ti, int tj, double* Li, double* Lj) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int base = kb + PB;
    const int i0 = base + ti * TB, j0 = base + tj * TB;
    for (int e = tid; e < TB * PB; e += LARGE_THREADS) {
        const int rr = e / PB, c = e % PB;      // consecutive threads: one row's panel entries
        const int ii = i0 + rr, jj = j0 + rr;
        Li[c * TBP + rr] = ii < n ? A[trow(ii) + kb + c] : 0.0;
        Lj[c * TBP + rr] = jj < n ? A[trow(jj) + kb + c] : 0.0;
    }
    __syncthreads();
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
#pragma unroll 4
    for (int c = 0; c < PB; ++c) {
        const double2 la = *(const double2*)&Li[c * TBP + ty * 4];
        const double2 lb = *(const double2*)&Li[c * TBP + ty * 4 + 2];
        const double2 ra = *(const double2*)&Lj[c * TBP + tx * 4];
        const double2 rb = *(const double2*)&Lj[c * TBP + tx * 4 + 2];
        const double li[4] = {la.x, la.y, lb.x, lb.y}, lj[4] = {ra.x, ra.y, rb.x, rb.y};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(li[a], lj[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = i0 + ty * 4 + a;
        if (i >= n) break;
        double* row = A + trow(i);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = j0 + tx * 4 + b;
            if (j <= i) row[j] -= acc[a][b];
        }
    }
    __syncthreads();
}

// L^T b = y (whole CTA, one row of L per step: row k removes b_k from r_0 .. r_{k-1}); b is
// written to w64 / w32; thread 0 returns sum b^2 and sum |b|
INFFT_D void back_solve(const double* __restrict__ A, double* __restrict__ r, int n, double* __restrict__ w64,
                        float* __restrict__ w32, double& bsq, double& babs) {
    const int tid = threadIdx.x;
    bsq = 0.0;
    babs = 0.0;
    for (int k = n - 1; k >= 0; --k) {
        const double* row = A + trow(k);
        const double bk = r[k] * row[k];
        for (int i = tid; i < k; i += blockDim.x) r[i] = fma(-row[i], bk, r[i]);
        if (tid == 0) {
            w64[k] = bk;
            w32[k] = (float)bk;
            bsq = fma(bk, bk, bsq);
            babs += fabs(bk);
        }
        __syncthreads();
    }
}

size_t large_smem(int nmax) { return (size_t)nmax * (sizeof(NodeK) + sizeof(double)); }

// one CTA per column of 129 .. GIANT_N nodes, largest first (atomic ticket), two CTAs per SM
__global__ void __launch_bounds__(LARGE_THREADS, 2)
k2_solve_large(const double2* __restrict__ x, const int32_t* __restrict__ col_off, const int32_t* __restrict__ col_node,
               const int32_t* __restrict__ order, int Ms1, int Ms2, K2 kp, double mu0, double* __restrict__ scratch,
               size_t slot_doubles, int32_t* __restrict__ ticket, double* __restrict__ w64, float* __restrict__ w32,
               double* __restrict__ J, uint8_t* __restrict__ wide, int32_t* __restrict__ counters, int nmax) {
    extern __shared__ __align__(16) double sm2[];
    NodeK* xl = (NodeK*)sm2;                     // nmax nodes of the column with their phases
    double* r = (double*)(xl + nmax);            // nmax
    __shared__ __align__(16) double Li[PB * TBP], Lj[PB * TBP];
    __shared__ PanelShared ps;
    __shared__ int s_job;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = LARGE_THREADS / 32;
    double* A = scratch + (size_t)blockIdx.x * slot_doubles;
    const int count = counters[C2_LIST0 + 3];
    for (;;) {
        if (tid == 0) s_job = atomicAdd(ticket, 1);
        __syncthreads();
        const int job = s_job;
        if (job >= count) break;
        const int p = order[job];
        const int off = col_off[p], n = col_off[p + 1] - off;
        const NodeK cp = column_point(p, Ms1, Ms2, kp);
        for (int i = tid; i < n; i += LARGE_THREADS) xl[i] = node_k(x[col_node[off + i]], kp);
        __syncthreads();
        double mu = mu0;
        bool ok = false;
        for (int attempt = 0; attempt < 3 && !ok; ++attempt) {
            for (int i = warp; i < n; i += NW) {       // one warp per row: coalesced stores
                const NodeK xi = xl[i];
                for (int j = lane; j <= i; j += 32) A[trow(i) + j] = (j == i) ? kp.diag + mu : re_kappa2(xi, xl[j], kp);
            }
            for (int i = tid; i < n; i += LARGE_THREADS) r[i] = re_kappa2(cp, xl[i], kp);
            if (tid == 0) { ps.fail = 0; ps.ysq = 0.0; }
            __syncthreads();
            for (int kb = 0; kb < n; kb += PB) {
                panel_step(A, r, n, kb, ps);
                if (ps.fail) break;
                const int nt = trailing_tiles(n, kb);
                for (int tile = 0; tile < nt; ++tile) {
                    int ti, tj;
                    tile_coords(tile, ti, tj);
                    trailing_tile(A, n, kb, ti, tj, Li, Lj);
                }
            }
            __syncthreads();
            ok = !ps.fail;
            if (!ok) mu *= 1e3;
            __syncthreads();
        }
        if (!ok) {
            for (int i = tid; i < n; i += LARGE_THREADS) { w64[off + i] = 0.0; w32[off + i] = 0.0f; }
            if (tid == 0) { J[p] = 1.0; atomicAdd(&counters[C2_FALLBACK], 1); }
            __syncthreads();
            continue;
        }
        if (tid == 0 && mu != mu0) atomicAdd(&counters[C2_FALLBACK], 1);
        double bsq, babs;
        back_solve(A, r, n, w64 + off, w32 + off, bsq, babs);
        if (tid == 0) {
            J[p] = 1.0 - ps.ysq - mu * bsq;
            const bool wd = babs > WIDE_COLUMN_L1;
            wide[p] = wd;
            if (wd) atomicAdd(&counters[C2_WIDE], 1);
        }
        __syncthreads();
    }
}

// ---- precompute: the largest columns, each spread over many CTAs -----------------
//
// Columns above GIANT_N nodes carry most of the Cholesky work (n^3/3) and would leave
// one SM busy long after the others.  They are factored together, one panel step per
// pair of launches: k2g_panel (one CTA per column) and k2g_update, whose grid walks the
// trailing tiles of all these columns as one flat index space (the per-step tile
// prefix over the columns is computed on the host from the column sizes).

struct GiantCol {
    int p, n, fail, pad;
    long long a_off;       // packed triangle in the giant scratch
    long long v_off;       // r (n doubles, padded to even), then the nodes (n NodeK)
    double ysq;
};

__global__ void __launch_bounds__(LARGE_THREADS) k2g_stage(const double2* __restrict__ x,
                                                           const int32_t* __restrict__ col_off,
                                                           const int32_t* __restrict__ col_node,
                                                           GiantCol* __restrict__ gs, double* __restrict__ gbase,
                                                           int Ms1, int Ms2, K2 kp) {
    GiantCol& g = gs[blockIdx.y];
    const int n = g.n, off = col_off[g.p];
    double* r = gbase + g.v_off;
    NodeK* xl = (NodeK*)(r + n + (n & 1));
    const NodeK cp = column_point(g.p, Ms1, Ms2, kp);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const NodeK v = node_k(x[col_node[off + i]], kp);
        xl[i] = v;
        r[i] = re_kappa2(cp, v, kp);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) { g.fail = 0; g.ysq = 0.0; }
}

// one warp per triangle row over all columns of the group (rows numbered through the
// exclusive prefix rowpre over the columns' sizes)
__global__ void __launch_bounds__(LARGE_THREADS) k2g_fill(const GiantCol* __restrict__ gs, double* __restrict__ gbase,
                                                          K2 kp, double mu, const int32_t* __restrict__ rowpre, int G) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (LARGE_THREADS / 32);
    const int total = rowpre[G];
    for (int t = blockIdx.x * (LARGE_THREADS / 32) + (threadIdx.x >> 5); t < total; t += nw) {
        int lo = 0, hi = G - 1;                            // last g with rowpre[g] <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (rowpre[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const GiantCol& g = gs[lo];
        const int n = g.n, i = t - rowpre[lo];
        double* A = gbase + g.a_off;
        const double* r = gbase + g.v_off;
        const NodeK* xl = (const NodeK*)(r + n + (n & 1));
        const NodeK xi = xl[i];
        for (int j = lane; j <= i; j += 32) A[trow(i) + j] = (j == i) ? kp.diag + mu : re_kappa2(xi, xl[j], kp);
    }
}

__global__ void __launch_bounds__(LARGE_THREADS) k2g_panel(GiantCol* __restrict__ gs, double* __restrict__ gbase,
                                                           int kb) {
    __shared__ PanelShared ps;
    GiantCol& g = gs[blockIdx.x];
    if (g.fail || kb >= g.n) return;                   // CTA-uniform
    if (threadIdx.x == 0) { ps.fail = 0; ps.ysq = g.ysq; }
    __syncthreads();
    panel_step(gbase + g.a_off, gbase + g.v_off, g.n, kb, ps);
    if (threadIdx.x == 0) { g.fail = ps.fail; g.ysq = ps.ysq; }
}

// prefix: G + 1 exclusive tile offsets of this step's trailing updates
__global__ void __launch_bounds__(LARGE_THREADS) k2g_update(const GiantCol* __restrict__ gs,
                                                            double* __restrict__ gbase, int kb,
                                                            const int32_t* __restrict__ prefix, int G) {
    __shared__ __align__(16) double Li[PB * TBP], Lj[PB * TBP];
    const int total = prefix[G];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int lo = 0, hi = G - 1;                            // last g with prefix[g] <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const GiantCol& g = gs[lo];
        if (g.fail) continue;                              // CTA-uniform
        int ti, tj;
        tile_coords(t - prefix[lo], ti, tj);
        trailing_tile(gbase + g.a_off, g.n, kb, ti, tj, Li, Lj);
    }
}

__global__ void __launch_bounds__(LARGE_THREADS) k2g_back(const GiantCol* __restrict__ gs, double* __restrict__ gbase,
                                                          const int32_t* __restrict__ col_off, double mu, int retried,
                                                          double* __restrict__ w64, float* __restrict__ w32,
                                                          double* __restrict__ J, uint8_t* __restrict__ wide,
                                                          int32_t* __restrict__ counters) {
    const GiantCol& g = gs[blockIdx.x];
    if (g.fail) return;                                    // retried by the host with a larger mu
    const int off = col_off[g.p];
    double bsq, babs;
    back_solve(gbase + g.a_off, gbase + g.v_off, g.n, w64 + off, w32 + off, bsq, babs);
    if (threadIdx.x == 0) {
        J[g.p] = 1.0 - g.ysq - mu * bsq;
        const bool wd = babs > WIDE_COLUMN_L1;
        wide[g.p] = wd;
        if (wd) atomicAdd(&counters[C2_WIDE], 1);
        if (retried) atomicAdd(&counters[C2_FALLBACK], 1);
    }
}

// columns that failed every attempt: b_l = 0, J_l = 1, counted
__global__ void k2g_give_up(const GiantCol* __restrict__ gs, const int32_t* __restrict__ col_off,
                            double* __restrict__ w64, float* __restrict__ w32, double* __restrict__ J,
                            int32_t* __restrict__ counters) {
    const GiantCol& g = gs[blockIdx.x];
    if (!g.fail) return;
    const int off = col_off[g.p];
    for (int i = threadIdx.x; i < g.n; i += blockDim.x) { w64[off + i] = 0.0; w32[off + i] = 0.0f; }
    if (threadIdx.x == 0) { J[g.p] = 1.0; atomicAdd(&counters[C2_FALLBACK], 1); }
}

// ---- apply ---------------------------------------------------------------------

// The fp32 spread reads no node index per entry.  The entries of column (a1, a2) are
// the nodes of I(l) in candidate order: the cells (a1 + d1, a2 - m .. a2 + m) for
// d1 = -m .. m, sorted nodes inside each, filtered by the exact test of eq:set_xj.  That
// test keeps every node of the cells with c_t in [a_t - m, a_t + m - 1] and, of the cells
// with c_t = a_t + m, only nodes with an integer u_t = fl(M_sigma,t x_t).  A column with no
// such node (nearly all: an integer u_t needs a node on a grid line) is therefore 2m
// cell-row runs of consecutive sorted nodes, d1 = -m .. m - 1, each the cells a2 - m ..
// a2 + m - 1 (two runs where they wrap), whose bounds the spread reads from cell_start
// (L2-resident) and whose node values it reads from the sorted copy of f.  The others are
// spread through their node indices.  Column kinds: bit 0 wide (||b_l||_1 > 32: float-float
// on the fp32 pipe), bit 1 indexed.
constexpr int K2_WIDE = 1, K2_INDEXED = 2;
constexpr int K2_RUNS_MAX = 64;   // 2m rows, two runs each where they wrap: m <= 16

// the cell ranges [c0[r], c1[r]] of the runs of a row (nr = 1, or 2 where a2 - m .. a2 + m - 1
// wraps); returns nr
INFFT_D int k2_row_ranges(int a2, int m, int Ms2, int (&c0)[2], int (&c1)[2]) {
    const int lo = a2 - m, hi = a2 + m - 1;
    if (lo < 0) { c0[0] = lo + Ms2; c1[0] = Ms2 - 1; c0[1] = 0; c1[1] = hi; return 2; }
    if (hi >= Ms2) { c0[0] = lo; c1[0] = Ms2 - 1; c0[1] = 0; c1[1] = hi - Ms2; return 2; }
    c0[0] = lo; c1[0] = hi;
    return 1;
}

// sorted-node range [s, e) of run j (row d1 = -m + j / nr, range j % nr) of column (a1, .)
INFFT_D void k2_run_bounds(const int32_t* __restrict__ cell_start, int Ms1, int Ms2, int a1, int m, int nr,
                           const int (&c0)[2], const int (&c1)[2], int j, int& s, int& e) {
    int r1 = a1 - m + j / nr;
    if (r1 < 0) r1 += Ms1;
    else if (r1 >= Ms1) r1 -= Ms1;
    const int r = j % nr;
    const int base = r1 * Ms2;
    s = cell_start[base + c0[r]];
    e = cell_start[base + c1[r] + 1];
}

// Low parts of the weights, fp32(b - fp32(b)), for the float-float spread of wide columns
__global__ void k2_lowparts(const float* __restrict__ w32, const double* __restrict__ w64, int nnz,
                            float* __restrict__ wlo) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x)
        wlo[e] = (float)(w64[e] - (double)w32[e]);
}

// The kind of every column (after the weights are final): a run column when its 2m runs
// hold exactly its |I(l)| entries
__global__ void k2_kinds(const int32_t* __restrict__ cell_start, const int32_t* __restrict__ col_off,
                         const uint8_t* __restrict__ wide, int Ms1, int Ms2, int m, int P,
                         uint8_t* __restrict__ kind, int32_t* __restrict__ counters) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const int a1 = p / Ms2, a2 = p - a1 * Ms2;
        int c0[2], c1[2];
        const int nr = k2_row_ranges(a2, m, Ms2, c0, c1);
        int cnt = 0;
        for (int j = 0; j < 2 * m * nr; ++j) {
            int sj, ej;
            k2_run_bounds(cell_start, Ms1, Ms2, a1, m, nr, c0, c1, j, sj, ej);
            cnt += ej - sj;
        }
        const bool runs = m <= K2_RUNS_MAX / 4 && cnt == col_off[p + 1] - col_off[p];
        kind[p] = (uint8_t)((wide[p] ? K2_WIDE : 0) | (runs ? 0 : K2_INDEXED));
        if (!runs) atomicAdd(&counters[C2_INDEXED], 1);
    }
}

// f in the order of the sorted nodes: fs[i] = f[perm[i]]
__global__ void k2_sort_values(const float2* __restrict__ f, const int32_t* __restrict__ perm, int N,
                               float2* __restrict__ fs) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) fs[i] = f[perm[i]];
}

// The run table of column (a1, a2) built by warp 0 of a CTA: rt[j] = (first sorted node,
// first entry) of run j, rt[R] = (0, number of entries).  Returns R.
INFFT_D int k2_build_runs(const int32_t* __restrict__ cell_start, int Ms1, int Ms2, int a1, int a2, int m, int lane,
                          int2* rt) {
    int c0[2], c1[2];
    const int nr = k2_row_ranges(a2, m, Ms2, c0, c1);
    const int R = 2 * m * nr;
    int run = 0;
    for (int j0 = 0; j0 < R; j0 += 32) {
        const int j = j0 + lane;
        int sj = 0, ej = 0;
        if (j < R) k2_run_bounds(cell_start, Ms1, Ms2, a1, m, nr, c0, c1, j, sj, ej);
        const int len = ej - sj;
        int inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (j < R) rt[j] = make_int2(sj, run + inc - len);
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) rt[R] = make_int2(0, run);
    return R;
}

// s + e = a + b exactly (Knuth's two-sum; the _rn intrinsics keep the compiler from
// reassociating or contracting)
INFFT_D void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// A thread's partial sum of a column: fp32 (four accumulator pairs, one per unrolled
// entry) or float-float ((s, c) pairs through two-sum, each product split exactly by an
// FMA: about 44 significant bits on the fp32 pipe, which runs 64 times as many lanes per
// clock as the fp64 pipe).
template <bool WIDE> struct K2Acc;

template <> struct K2Acc<false> {
    float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
    INFFT_D void add(int u, float w, float, float2 v) {
        ar[u] = fmaf(w, v.x, ar[u]);
        ai[u] = fmaf(w, v.y, ai[u]);
    }
    INFFT_D float4 total() const {
        return make_float4((ar[0] + ar[1]) + (ar[2] + ar[3]), 0.f, (ai[0] + ai[1]) + (ai[2] + ai[3]), 0.f);
    }
};

template <> struct K2Acc<true> {
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    INFFT_D void add(int, float wh, float wl, float2 v) {
        const float tr = __fmul_rn(wh, v.x), ti = __fmul_rn(wh, v.y);
        const float lr = fmaf(wl, v.x, fmaf(wh, v.x, -tr)), li = fmaf(wl, v.y, fmaf(wh, v.y, -ti));
        float t, err;
        two_sum(sr, tr, t, err);
        sr = t;
        cr += err + lr;
        two_sum(si, ti, t, err);
        si = t;
        ci += err + li;
    }
    INFFT_D float4 total() const { return make_float4(sr, cr, si, ci); }
};

// (s, c) pairs of two float-float sums combined (plain sums: c = 0 stays 0)
template <bool WIDE> INFFT_D float4 k2_combine(float4 a, float4 b) {
    if (!WIDE) return make_float4(a.x + b.x, 0.f, a.z + b.z, 0.f);
    float t, err;
    two_sum(a.x, b.x, t, err);
    a.x = t;
    a.y += b.y + err;
    two_sum(a.z, b.z, t, err);
    a.z = t;
    a.w += b.w + err;
    return a;
}

template <bool WIDE> INFFT_D float4 k2_reduce(unsigned mask, float4 v, int width) {
    for (int o = width / 2; o; o >>= 1) {
        const float4 u = make_float4(__shfl_xor_sync(mask, v.x, o), WIDE ? __shfl_xor_sync(mask, v.y, o) : 0.f,
                                     __shfl_xor_sync(mask, v.z, o), WIDE ? __shfl_xor_sync(mask, v.w, o) : 0.f);
        v = k2_combine<WIDE>(v, u);
    }
    return v;
}

// entries o0, o0 + step, .. < len of one run (weights w, low parts wl, node values v), four
// loads in flight
template <bool WIDE>
INFFT_D void k2_sum_run(K2Acc<WIDE>& acc, const float* __restrict__ w, const float* __restrict__ wl,
                        const float2* __restrict__ v, int o0, int step, int len) {
    int o = o0;
    for (; o + 3 * step < len; o += 4 * step) {
        float wq[4], lq[4];
        float2 vq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            wq[u] = w[o + u * step];
            lq[u] = WIDE ? wl[o + u * step] : 0.f;
            vq[u] = v[o + u * step];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc.add(u, wq[u], lq[u], vq[u]);
    }
    for (; o < len; o += step) acc.add(0, w[o], WIDE ? wl[o] : 0.f, v[o]);
}

// entries q = q0, q0 + step, .. < n of an indexed column (node values through node[q])
template <bool WIDE>
INFFT_D void k2_sum_indexed(K2Acc<WIDE>& acc, const float* __restrict__ w, const float* __restrict__ wl,
                            const float2* __restrict__ f, const int32_t* __restrict__ node, int q0, int step, int n) {
    int q = q0;
    for (; q + 3 * step < n; q += 4 * step) {
        int nq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) nq[u] = node[q + u * step];
        float wq[4], lq[4];
        float2 vq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            wq[u] = w[q + u * step];
            lq[u] = WIDE ? wl[q + u * step] : 0.f;
            vq[u] = f[nq[u]];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc.add(u, wq[u], lq[u], vq[u]);
    }
    for (; q < n; q += step) acc.add(0, w[q], WIDE ? wl[q] : 0.f, f[node[q]]);
}

// One column by a group of LPC lanes (sub = lane in the group).  Run columns: lane sub takes
// runs sub, sub + LPC, .. whole (their first entries from a scan of the run lengths over the
// group), so a lane's loads walk consecutive weights and consecutive sorted node values;
// indexed columns: the lanes walk the entries LPC apart.  Returns the group's total on every lane.
template <int LPC, bool WIDE>
INFFT_D float4 k2_column_group(int p, int sub, unsigned mask, int s, int n, bool runs, const float2* __restrict__ f,
                               const float2* __restrict__ fs, const int32_t* __restrict__ cell_start,
                               const int32_t* __restrict__ col_node, const float* __restrict__ w32,
                               const float* __restrict__ wlo, int Ms1, int Ms2, int m) {
    K2Acc<WIDE> acc;
    const float* w = w32 + s;
    const float* wl = wlo + s;
    if (runs) {
        const int a1 = p / Ms2, a2 = p - a1 * Ms2;
        int c0[2], c1[2];
        const int nr = k2_row_ranges(a2, m, Ms2, c0, c1);
        const int R = 2 * m * nr;
        int base = 0;
        for (int j0 = 0; j0 < R; j0 += LPC) {
            const int j = j0 + sub;
            int sj = 0, ej = 0;
            if (j < R) k2_run_bounds(cell_start, Ms1, Ms2, a1, m, nr, c0, c1, j, sj, ej);
            const int len = ej - sj;
            int inc = len;
#pragma unroll
            for (int o = 1; o < LPC; o <<= 1) {
                const int v = __shfl_up_sync(mask, inc, o, LPC);
                if (sub >= o) inc += v;
            }
            const int eo = base + inc - len;
            base += __shfl_sync(mask, inc, LPC - 1, LPC);
            k2_sum_run<WIDE>(acc, w + eo, wl + eo, fs + sj, 0, 1, len);
        }
    } else {
        k2_sum_indexed<WIDE>(acc, w, wl, f, col_node + s, sub, LPC, n);
    }
    return k2_reduce<WIDE>(mask, acc.total(), LPC);
}

// One column by a CTA of 256 threads (columns above SPREAD_BIG entries): run columns take the
// runs one after another, all threads over each run's entries.
template <bool WIDE>
INFFT_D float4 k2_column_cta(int p, int s, int n, bool runs, const float2* __restrict__ f,
                             const float2* __restrict__ fs, const int32_t* __restrict__ cell_start,
                             const int32_t* __restrict__ col_node, const float* __restrict__ w32,
                             const float* __restrict__ wlo, int Ms1, int Ms2, int m, int2* rt, float4* red) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    K2Acc<WIDE> acc;
    const float* w = w32 + s;
    const float* wl = wlo + s;
    if (runs) {
        const int a1 = p / Ms2, a2 = p - a1 * Ms2;
        if (warp == 0) k2_build_runs(cell_start, Ms1, Ms2, a1, a2, m, lane, rt);
        int c0[2], c1[2];
        const int R = 2 * m * k2_row_ranges(a2, m, Ms2, c0, c1);
        __syncthreads();
        for (int j = 0; j < R; ++j) {
            const int2 r = rt[j];
            k2_sum_run<WIDE>(acc, w + r.y, wl + r.y, fs + r.x, tid, 256, rt[j + 1].y - r.y);
        }
    } else {
        k2_sum_indexed<WIDE>(acc, w, wl, f, col_node + s, tid, 256, n);
    }
    const float4 v = k2_reduce<WIDE>(0xffffffffu, acc.total(), 32);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float4 t = red[0];
    for (int i = 1; i < 8; ++i) t = k2_combine<WIDE>(t, red[i]);
    return t;
}

// fp32 apply: g_p = sum_{e in column p} b_e f_{node(e)}, LPC lanes per column; columns above
// SPREAD_BIG entries (the first nbig CTAs, listed in big) take a whole CTA.  Ordinary columns:
// fp32 weights and accumulation; wide columns: float-float.
template <int LPC>
__global__ void __launch_bounds__(256, 6) k2_spread32(const float2* __restrict__ f, const float2* __restrict__ fs,
                                                   const int32_t* __restrict__ col_off,
                                                   const int32_t* __restrict__ cell_start,
                                                   const int32_t* __restrict__ col_node, const float* __restrict__ w32,
                                                   const float* __restrict__ wlo, const uint8_t* __restrict__ kind,
                                                   int Ms1, int Ms2, int m, int P, float2* __restrict__ g,
                                                   const int32_t* __restrict__ big, int nbig) {
    __shared__ int2 rt[K2_RUNS_MAX + 1];
    __shared__ float4 red[8];
    if ((int)blockIdx.x < nbig) {                          // a column above SPREAD_BIG entries
        const int p = big[blockIdx.x];
        const int s = col_off[p], n = col_off[p + 1] - s;
        const int k = kind[p];
        const bool runs = !(k & K2_INDEXED);
        const float4 t = (k & K2_WIDE)
            ? k2_column_cta<true>(p, s, n, runs, f, fs, cell_start, col_node, w32, wlo, Ms1, Ms2, m, rt, red)
            : k2_column_cta<false>(p, s, n, runs, f, fs, cell_start, col_node, w32, wlo, Ms1, Ms2, m, rt, red);
        if (threadIdx.x == 0) g[p] = make_float2(t.x + t.y, t.z + t.w);
        return;
    }
    const int sub = threadIdx.x & (LPC - 1);
    const int p = (blockIdx.x - nbig) * (256 / LPC) + threadIdx.x / LPC;
    const unsigned mask = LPC == 32 ? 0xffffffffu : ((1u << LPC) - 1) << ((threadIdx.x & 31) & ~(LPC - 1));
    if (p >= P) return;                                    // uniform over the column's lanes
    const int s = col_off[p], n = col_off[p + 1] - s;
    if (n > SPREAD_BIG) return;                            // spread by its own CTA
    const int k = kind[p];
    const bool runs = !(k & K2_INDEXED);
    const float4 t = (k & K2_WIDE)
        ? k2_column_group<LPC, true>(p, sub, mask, s, n, runs, f, fs, cell_start, col_node, w32, wlo, Ms1, Ms2, m)
        : k2_column_group<LPC, false>(p, sub, mask, s, n, runs, f, fs, cell_start, col_node, w32, wlo, Ms1, Ms2, m);
    if (sub == 0) g[p] = make_float2(t.x + t.y, t.z + t.w);
}

// fp64 apply: fp64 weights, inputs and accumulation, one warp per column
__global__ void __launch_bounds__(256) k2_spread64(const double2* __restrict__ f, const int32_t* __restrict__ col_off,
                                                   const int32_t* __restrict__ col_node,
                                                   const double* __restrict__ w64, int P, double2* __restrict__ g) {
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (p >= P) return;
    const int s = col_off[p], e = col_off[p + 1];
    double ar = 0.0, ai = 0.0;
    for (int q = s + lane; q < e; q += 32) {
        const double w = w64[q];
        const double2 v = f[col_node[q]];
        ar = fma(w, v.x, ar);
        ai = fma(w, v.y, ai);
    }
    for (int o = 16; o; o >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) g[p] = make_double2(ar, ai);
}

// pass R: rows a1 in [a1_0, a1_0 + C) of the grid, transform over a2 (length Ms2), keep
// k2 = -M2/2 .. M2/2-1 with the factor (-1)^k2 and store Y[k2 + M2/2][a1]
template <typename T>
__global__ void __launch_bounds__(FFT2_THREADS) k2_fft_rows(const cplx_t<T>* __restrict__ g, cplx_t<T>* __restrict__ Y,
                                                            int log2, int Ms1, int M2, int C) {
    using Cx = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char fsm[];
    const int Ms2 = 1 << log2;
    Cx* a = (Cx*)fsm;
    Cx* b = a + C * Ms2;
    const int a1_0 = blockIdx.x * C;
    for (int t = threadIdx.x; t < C * Ms2; t += blockDim.x) a[t] = g[(size_t)a1_0 * Ms2 + t];
    __syncthreads();
    const Cx* res = smem_fft<T, -1>(a, b, log2, C);
    for (int t = threadIdx.x; t < C * M2; t += blockDim.x) {
        const int rr = t % C, kk = t / C;
        const int k2 = kk - M2 / 2;
        const Cx v = res[rr * Ms2 + (k2 & (Ms2 - 1))];
        Y[(size_t)kk * Ms1 + a1_0 + rr] = (k2 & 1) ? cmake(-v.x, -v.y) : v;
    }
}

// pass C: rows kk in [kk_0, kk_0 + C) of Y, transform over a1 (length Ms1), keep k1 and
// store fhat[k1 + M1/2][kk] = (-1)^k1 d_k * value (d_k = 1/(Ms1 Ms2), 0 for kernel sym
// when k1 = -M1/2 or k2 = -M2/2)
template <typename T>
__global__ void __launch_bounds__(FFT2_THREADS) k2_fft_cols(const cplx_t<T>* __restrict__ Y, cplx_t<T>* __restrict__ fhat,
                                                            int log1, int M1, int M2, int C, T inv, int sym) {
    using Cx = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char fsm[];
    const int Ms1 = 1 << log1;
    Cx* a = (Cx*)fsm;
    Cx* b = a + C * Ms1;
    const int kk_0 = blockIdx.x * C;
    for (int t = threadIdx.x; t < C * Ms1; t += blockDim.x) a[t] = Y[(size_t)kk_0 * Ms1 + t];
    __syncthreads();
    const Cx* res = smem_fft<T, -1>(a, b, log1, C);
    for (int t = threadIdx.x; t < C * M1; t += blockDim.x) {
        const int rr = t % C, k1i = t / C;
        const int k1 = k1i - M1 / 2;
        const int kk = kk_0 + rr;
        T d = (k1 & 1) ? -inv : inv;
        if (sym && (k1 == -M1 / 2 || kk == 0)) d = (T)0;
        const Cx v = res[rr * Ms1 + (k1 & (Ms1 - 1))];
        fhat[(size_t)k1i * M2 + kk] = cmake(v.x * d, v.y * d);
    }
}

int fft_batch(int logn) { return std::max(1, 2048 >> logn); }

template <typename K> cudaError_t smem_attr(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

K2 kernel_params(const infft2d_plan_s* p) {
    K2 k;
    k.M1 = (double)p->M1;
    k.M2 = (double)p->M2;
    k.sym = p->kernel == INFFT_KERNEL_SYM;
    k.K1 = k.sym ? k.M1 - 1.0 : k.M1;
    k.K2 = k.sym ? k.M2 - 1.0 : k.M2;
    k.inv = 1.0 / ((double)p->Ms1 * (double)p->Ms2);
    k.diag = k.K1 * k.K2 * k.inv;
    // node differences within a column are at most (2m + 1)/M_sigma,t per dimension
    const double a1 = 3.141592653589793 * (2.0 * p->m + 1.0) / (double)p->Ms1;
    const double a2 = 3.141592653589793 * (2.0 * p->m + 1.0) / (double)p->Ms2;
    k.shortd = a1 <= 0.25 && a2 <= 0.25;
    return k;
}

struct Carver2 {
    char* base = nullptr;
    size_t off = 0;
    template <typename X> void take(X*& ptr, size_t count) {
        off = (off + 255) & ~(size_t)255;
        ptr = base ? (X*)(base + off) : nullptr;
        off += count * sizeof(X) + 16;
    }
};

void layout2(infft2d_plan_s* p, Carver2& c) {
    const size_t N = p->N, P = p->P, M = p->M1 * p->M2;
    c.take(p->x, N); c.take(p->xs, N); c.take(p->node_cell, N); c.take(p->perm, N);
    c.take(p->cell_start, P + 1); c.take(p->cursor, P); c.take(p->big_cells, P);
    c.take(p->col_off, P + 1); c.take(p->col_node, p->nnz_cap);
    c.take(p->lists, 5 * P); c.take(p->order, P); c.take(p->spread_big, P); c.take(p->hist, LARGE_NMAX + 2);
    c.take(p->counters, C2_N);
    c.take(p->w32, p->nnz_cap); c.take(p->w64, p->nnz_cap); c.take(p->wlo, p->nnz_cap); c.take(p->J, P); c.take(p->wide, P);
    c.take(p->kind, P); c.take(p->fsort, N);
    double2 *grid, *work, *si, *so;
    c.take(grid, P); c.take(work, (size_t)p->M2 * p->Ms1);
    const size_t stage = std::max(N, M);
    c.take(si, stage); c.take(so, stage);
    p->grid = grid; p->work = work; p->stage_in = si; p->stage_out = so;
}

cudaError_t run_pattern2(infft2d_plan_s* p, cudaStream_t s) {
    const int N = (int)p->N, P = (int)p->P, Ms1 = (int)p->Ms1, Ms2 = (int)p->Ms2;
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->counters, 0, C2_N * sizeof(int32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p->cell_start, 0, (P + 1) * sizeof(int32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p->cursor, 0, P * sizeof(int32_t), s)) != cudaSuccess) return e;
    const int nb = (N + 255) / 256, pb = (P + 255) / 256;
    k2_cells<<<nb, 256, 0, s>>>(p->x, N, Ms1, Ms2, p->node_cell, p->cell_start, p->counters);
    k2_scan<<<1, 1024, 0, s>>>(p->cell_start, P);
    k2_scatter<<<nb, 256, 0, s>>>(p->node_cell, N, p->cell_start, p->cursor, p->perm);
    k2_cell_sort<<<pb, 256, 0, s>>>(p->cell_start, P, p->perm, p->big_cells, p->counters);
    k2_cell_sort_big<<<256, 256, 0, s>>>(p->cell_start, p->perm, p->big_cells, p->counters);
    k2_gather_nodes<<<nb, 256, 0, s>>>(p->x, p->perm, p->cell_start, P, p->xs);
    const int cb = (P + 7) / 8;
    k2_columns<false><<<cb, 256, 0, s>>>(p->xs, p->perm, p->cell_start, Ms1, Ms2, p->m, p->col_off, nullptr,
                                         nullptr, p->counters);
    k2_scan<<<1, 1024, 0, s>>>(p->col_off, P);
    k2_columns<true><<<cb, 256, 0, s>>>(p->xs, p->perm, p->cell_start, Ms1, Ms2, p->m, nullptr, p->col_off,
                                        p->col_node, p->counters);
    count_launches(9);
    return cudaGetLastError();
}

// The columns above GIANT_N nodes (list 4): groups whose triangles fit GIANT_BUDGET are
// factored together, one panel step per (k2g_panel, k2g_update) pair of launches; a group's
// columns whose Cholesky failed are retried with mu raised 1000-fold, twice.
cudaError_t run_giants(infft2d_plan_s* p, int G, const K2& kp, double mu, int sms, cudaStream_t s) {
    cudaError_t e;
    std::vector<int32_t> list(G), off(p->P + 1);
    if ((e = cudaMemcpy(list.data(), p->lists + 4 * p->P, G * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpy(off.data(), p->col_off, (p->P + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    std::sort(list.begin(), list.end());
    std::vector<std::vector<GiantCol>> groups(1);
    size_t used = 0, need = 0;
    for (int q : list) {
        GiantCol g = {};
        g.p = q;
        g.n = off[q + 1] - off[q];
        const size_t tri = ((size_t)g.n * (g.n + 1) / 2 + 1) & ~(size_t)1;
        const size_t vec = ((size_t)7 * g.n + 3) & ~(size_t)1;   // r, the nodes (6 doubles each); even: 16-byte alignment
        if (!groups.back().empty() && (used + tri + vec) * sizeof(double) > GIANT_BUDGET) {
            groups.emplace_back();
            used = 0;
        }
        g.a_off = (long long)used;
        g.v_off = (long long)(used + tri);
        used += tri + vec;
        need = std::max(need, used);
        groups.back().push_back(g);
    }
    if (p->gscratch_doubles < need) {
        if (p->gscratch) cudaFree(p->gscratch);
        p->gscratch = nullptr;
        p->gscratch_doubles = 0;
        if ((e = cudaMalloc(&p->gscratch, need * sizeof(double))) != cudaSuccess) return e;
        p->gscratch_doubles = need;
    }
    size_t gmax = 0;
    for (auto& grp : groups) gmax = std::max(gmax, grp.size());
    if (p->gdesc_cap < (int)gmax) {
        if (p->gdesc) cudaFree(p->gdesc);
        p->gdesc = nullptr;
        p->gdesc_cap = 0;
        if ((e = cudaMalloc(&p->gdesc, gmax * sizeof(GiantCol))) != cudaSuccess) return e;
        p->gdesc_cap = (int)gmax;
    }
    GiantCol* gd = (GiantCol*)p->gdesc;
    for (auto grp : groups) {
        for (int attempt = 0; attempt < 3 && !grp.empty(); ++attempt) {
            const int Gg = (int)grp.size();
            const double mu_a = mu * std::pow(1e3, attempt);
            int nmax = 0;
            for (auto& g : grp) nmax = std::max(nmax, g.n);
            const int steps = (nmax + PB - 1) / PB;
            std::vector<int32_t> prefix((size_t)(steps + 1) * (Gg + 1));
            for (int st = 0; st < steps; ++st) {
                int32_t run = 0;
                for (int i = 0; i < Gg; ++i) {
                    prefix[(size_t)st * (Gg + 1) + i] = run;
                    run += trailing_tiles(grp[i].n, st * PB);
                }
                prefix[(size_t)st * (Gg + 1) + Gg] = run;
            }
            int32_t* rowpre = &prefix[(size_t)steps * (Gg + 1)];   // triangle rows of the group's columns
            int32_t rows = 0;
            for (int i = 0; i < Gg; ++i) {
                rowpre[i] = rows;
                rows += grp[i].n;
            }
            rowpre[Gg] = rows;
            if (p->gprefix_cap < prefix.size()) {
                if (p->gprefix) cudaFree(p->gprefix);
                p->gprefix = nullptr;
                p->gprefix_cap = 0;
                if ((e = cudaMalloc(&p->gprefix, prefix.size() * sizeof(int32_t))) != cudaSuccess) return e;
                p->gprefix_cap = prefix.size();
            }
            if ((e = cudaMemcpy(gd, grp.data(), Gg * sizeof(GiantCol), cudaMemcpyHostToDevice)) != cudaSuccess)
                return e;
            if ((e = cudaMemcpy(p->gprefix, prefix.data(), prefix.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
                return e;
            const int xs = std::max(1, std::min((nmax + 255) / 256, (4 * sms + Gg - 1) / Gg));
            k2g_stage<<<dim3(xs, Gg), LARGE_THREADS, 0, s>>>(p->x, p->col_off, p->col_node, gd, p->gscratch,
                                                            (int)p->Ms1, (int)p->Ms2, kp);
            k2g_fill<<<std::min((rows + 7) / 8, 16 * sms), LARGE_THREADS, 0, s>>>(
                gd, p->gscratch, kp, mu_a, p->gprefix + (size_t)steps * (Gg + 1), Gg);
            int launches = 2;
            for (int st = 0; st < steps; ++st) {
                k2g_panel<<<Gg, LARGE_THREADS, 0, s>>>(gd, p->gscratch, st * PB);
                const int tiles = prefix[(size_t)st * (Gg + 1) + Gg];
                if (tiles > 0)
                    k2g_update<<<std::min(tiles, 4 * sms), LARGE_THREADS, 0, s>>>(
                        gd, p->gscratch, st * PB, p->gprefix + (size_t)st * (Gg + 1), Gg);
                launches += 1 + (tiles > 0);
            }
            k2g_back<<<Gg, LARGE_THREADS, 0, s>>>(gd, p->gscratch, p->col_off, mu_a, attempt > 0, p->w64, p->w32,
                                                  p->J, p->wide, p->counters);
            count_launches(launches + 1);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            std::vector<GiantCol> back(Gg);
            if ((e = cudaMemcpyAsync(back.data(), gd, Gg * sizeof(GiantCol), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            std::vector<GiantCol> failed;
            for (auto& g : back)
                if (g.fail) failed.push_back(g);
            if (!failed.empty() && attempt == 2) {
                if ((e = cudaMemcpy(gd, failed.data(), failed.size() * sizeof(GiantCol), cudaMemcpyHostToDevice)) !=
                    cudaSuccess)
                    return e;
                k2g_give_up<<<(int)failed.size(), 256, 0, s>>>(gd, p->col_off, p->w64, p->w32, p->J, p->counters);
                count_launches(1);
            }
            grp = failed;
        }
    }
    return cudaGetLastError();
}

cudaError_t run_precompute2(infft2d_plan_s* p, cudaStream_t s) {
    const int P = (int)p->P, Ms1 = (int)p->Ms1, Ms2 = (int)p->Ms2;
    const K2 kp = kernel_params(p);
    const double mu = p->tau * kp.diag;
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->counters + C2_FALLBACK, 0, 2 * sizeof(int32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p->counters + C2_LIST0, 0, 5 * sizeof(int32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p->counters + C2_WIDE, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p->counters + C2_INDEXED, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p->hist, 0, (LARGE_NMAX + 2) * sizeof(int32_t), s)) != cudaSuccess) return e;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device)) != cudaSuccess) return e;
    if (sms <= 0) return cudaErrorInvalidDevice;
    if ((e = cudaMemsetAsync(p->counters + C2_SPREAD_BIG, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    k2_route<<<(P + 255) / 256, 256, 0, s>>>(p->col_off, P, p->lists, p->w64, p->w32, p->J, p->wide, p->hist,
                                             p->spread_big, p->counters);
    count_launches(1);
    // the list lengths and the columns for the multi-CTA solver decide the launches below
    int32_t cnt[C2_N];
    if ((e = cudaMemcpyAsync(cnt, p->counters, sizeof cnt, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    const int G = cnt[C2_LIST0 + 4];
    p->spread_big_count = cnt[C2_SPREAD_BIG];
    // shared-memory tiers
    auto t0 = k2_solve_small<32>;
    auto t1 = k2_solve_small<64>;
    auto t2 = k2_solve_small<128>;
    const size_t s0 = small_smem<32>(), s1 = small_smem<64>(), s2 = small_smem<128>();
    if ((e = smem_attr(t0, s0)) != cudaSuccess) return e;
    if ((e = smem_attr(t1, s1)) != cudaSuccess) return e;
    if ((e = smem_attr(t2, s2)) != cudaSuccess) return e;
    int o0 = 1, o1 = 1, o2 = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o0, t0, 32, s0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, t1, 64, s1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, t2, 128, s2);
    if (cnt[C2_LIST0 + 0])
        t0<<<std::max(o0, 1) * sms, 32, s0, s>>>(p->x, p->col_off, p->col_node, p->lists, 0, Ms1, Ms2, kp, mu,
                                                  p->w64, p->w32, p->J, p->wide, p->counters);
    if (cnt[C2_LIST0 + 1])
        t1<<<std::max(o1, 1) * sms, 64, s1, s>>>(p->x, p->col_off, p->col_node, p->lists + P, 1, Ms1, Ms2, kp, mu,
                                                  p->w64, p->w32, p->J, p->wide, p->counters);
    if (cnt[C2_LIST0 + 2])
        t2<<<std::max(o2, 1) * sms, 128, s2, s>>>(p->x, p->col_off, p->col_node, p->lists + 2 * P, 2, Ms1, Ms2, kp,
                                                   mu, p->w64, p->w32, p->J, p->wide, p->counters);
    count_launches(3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // one CTA per column of 129 .. GIANT_N nodes
    if (cnt[C2_LIST0 + 3]) {
        // the shared-memory layout keeps 16-byte alignment with an even nmax
        const int nmax = (std::min(p->max_column, GIANT_N) + 1) & ~1;
        const size_t slot = (size_t)nmax * (nmax + 1) / 2;
        const int slots = std::max(1, std::min(2 * sms, cnt[C2_LIST0 + 3]));   // two CTAs per SM
        if (p->scratch_doubles < slot * slots) {
            if (p->scratch) cudaFree(p->scratch);
            p->scratch = nullptr;
            p->scratch_doubles = 0;
            if ((e = cudaMalloc(&p->scratch, slot * slots * sizeof(double))) != cudaSuccess) return e;
            p->scratch_doubles = slot * slots;
        }
        k2_scan<<<1, 1024, 0, s>>>(p->hist, LARGE_NMAX + 1);
        k2_order_large<<<4 * sms, 256, 0, s>>>(p->col_off, p->lists + 3 * P, P, p->hist, p->order, p->counters);
        if ((e = cudaMemsetAsync(p->hist + LARGE_NMAX + 1, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
        const size_t sm = large_smem(nmax);
        if ((e = smem_attr(k2_solve_large, sm)) != cudaSuccess) return e;
        k2_solve_large<<<slots, LARGE_THREADS, sm, s>>>(p->x, p->col_off, p->col_node, p->order, Ms1, Ms2, kp, mu,
                                                        p->scratch, slot, p->hist + LARGE_NMAX + 1, p->w64, p->w32,
                                                        p->J, p->wide, p->counters, nmax);
        count_launches(3);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (G > 0 && (e = run_giants(p, G, kp, mu, sms, s)) != cudaSuccess) return e;
    if (p->nnz > 0) {
        k2_lowparts<<<(int)std::min<int64_t>((p->nnz + 255) / 256, 16 * sms), 256, 0, s>>>(p->w32, p->w64,
                                                                                       (int)p->nnz, p->wlo);
        count_launches(1);
    }
    k2_kinds<<<(int)std::min<int64_t>((P + 255) / 256, 16 * sms), 256, 0, s>>>(p->cell_start, p->col_off, p->wide,
                                                                              Ms1, Ms2, p->m, P, p->kind,
                                                                              p->counters);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T> cudaError_t run_apply2(infft2d_plan_s* p, const void* f, void* fhat, cudaStream_t s) {
    using Cx = cplx_t<T>;
    const int P = (int)p->P;
    Cx* g = (Cx*)p->grid;
    Cx* Y = (Cx*)p->work;
    if constexpr (sizeof(T) == 4) {
        const int N = (int)p->N;
        k2_sort_values<<<(N + 255) / 256, 256, 0, s>>>((const float2*)f, p->perm, N, p->fsort);
        k2_spread32<SPREAD_LPC><<<p->spread_big_count + (P + 256 / SPREAD_LPC - 1) / (256 / SPREAD_LPC), 256, 0, s>>>(
            (const float2*)f, p->fsort, p->col_off, p->cell_start, p->col_node, p->w32, p->wlo, p->kind,
            (int)p->Ms1, (int)p->Ms2, p->m, P, g, p->spread_big, p->spread_big_count);
        count_launches(2);
    } else {
        k2_spread64<<<(P + 7) / 8, 256, 0, s>>>((const double2*)f, p->col_off, p->col_node, p->w64, P, g);
        count_launches(1);
    }
    if constexpr (sizeof(T) == 4) {
        if (fft2d_r8_supported(p->log1, p->log2, (int)p->M2))
            return fft2d_adjoint_r8((const float2*)g, (float2*)Y, (float2*)fhat, p->log1, p->log2, (int)p->M1,
                                    (int)p->M2, p->kernel == INFFT_KERNEL_SYM, s);
    }
    const int C2 = std::min<int>(fft_batch(p->log2), (int)p->Ms1);
    const int C1 = std::min<int>(fft_batch(p->log1), (int)(p->M2 & -p->M2));   // a divisor of M2
    const size_t sm2 = 2 * (size_t)C2 * p->Ms2 * sizeof(Cx), sm1 = 2 * (size_t)C1 * p->Ms1 * sizeof(Cx);
    cudaError_t e;
    if ((e = smem_attr(k2_fft_rows<T>, sm2)) != cudaSuccess) return e;
    if ((e = smem_attr(k2_fft_cols<T>, sm1)) != cudaSuccess) return e;
    k2_fft_rows<T><<<(int)p->Ms1 / C2, FFT2_THREADS, sm2, s>>>(g, Y, p->log2, (int)p->Ms1, (int)p->M2, C2);
    k2_fft_cols<T><<<(int)p->M2 / C1, FFT2_THREADS, sm1, s>>>(Y, (Cx*)fhat, p->log1, (int)p->M1, (int)p->M2, C1,
                                                              (T)(1.0 / ((double)p->Ms1 * (double)p->Ms2)),
                                                              p->kernel == INFFT_KERNEL_SYM);
    count_launches(2);
    return cudaGetLastError();
}

int ilog2_exact(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return (int64_t(1) << l) == v ? l : -1;
}

template <typename T> infft_status apply2_impl(infft2d_plan_s* p, const T* f, T* fhat, infft_stream_t stream) {
    if (!p) return fail2(INFFT_EINVAL, "plan is NULL");
    if (!f || !fhat) return fail2(INFFT_EINVAL, "f and fhat must not be NULL");
    if (!p->precomputed) return fail2(INFFT_ENOTREADY, "infft2d_apply before infft2d_precompute");
    DeviceGuard2 g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    const size_t csz = 2 * sizeof(T);
    const int64_t M = p->M1 * p->M2;
    const void* fin = f;
    cudaError_t e;
    if (!on_device2(f)) {
        if ((e = cudaMemcpyAsync(p->stage_in, f, p->N * csz, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail2(e, "copy f to device");
        fin = p->stage_in;
    }
    const bool host_out = !on_device2(fhat);
    void* out = host_out ? p->stage_out : (void*)fhat;
    if ((e = run_apply2<T>(p, fin, out, s)) != cudaSuccess) return cuda_fail2(e, "apply");
    if (host_out) {
        if ((e = cudaMemcpyAsync(fhat, p->stage_out, M * csz, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail2(e, "copy fhat to host");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail2(e, "synchronize");
    }
    return INFFT_OK;
}

}  // namespace

extern "C" {

infft_status infft2d_plan_create(int64_t M1, int64_t M2, int64_t N, double sigma, int m, int kernel, double tau,
                                 infft2d_plan_t* out) {
    if (!out) return fail2(INFFT_EINVAL, "out is NULL");
    *out = nullptr;
    if (M1 < 2 || (M1 & 1) || M2 < 2 || (M2 & 1))
        return fail2(INFFT_EINVAL, "M1 and M2 must be even and >= 2 (got %lld, %lld)", (long long)M1, (long long)M2);
    if (N < 1) return fail2(INFFT_EINVAL, "N must be >= 1 (got %lld)", (long long)N);
    if (!std::isfinite(sigma) || sigma < 1.0) return fail2(INFFT_EINVAL, "sigma must be >= 1 (got %g)", sigma);
    if (kernel != INFFT_KERNEL_FULL && kernel != INFFT_KERNEL_SYM)
        return fail2(INFFT_EINVAL, "kernel must be INFFT_KERNEL_FULL or INFFT_KERNEL_SYM (got %d)", kernel);
    if (!(tau >= 0.0 && tau < 1.0)) return fail2(INFFT_EINVAL, "tau must be in [0, 1) (got %g)", tau);
    const double d1 = sigma * (double)M1, d2 = sigma * (double)M2;
    if (d1 != std::floor(d1) || d2 != std::floor(d2) || d1 > 4096.0 || d2 > 4096.0)
        return fail2(INFFT_EINVAL, "sigma*M_t must be integers (got %.17g, %.17g)", d1, d2);
    const int64_t Ms1 = (int64_t)d1, Ms2 = (int64_t)d2;
    const int l1 = ilog2_exact(Ms1), l2 = ilog2_exact(Ms2);
    if (l1 < 2 || l2 < 2 || Ms1 > 2048 || Ms2 > 2048)
        return fail2(INFFT_EUNSUPPORTED, "M_sigma,t = sigma M_t must be powers of two in [4, 2048] (got %lld, %lld)",
                     (long long)Ms1, (long long)Ms2);
    if (m < 1 || 2 * (int64_t)m >= Ms1 || 2 * (int64_t)m >= Ms2)
        return fail2(INFFT_EINVAL, "need m >= 1 and 2m < M_sigma,t (m = %d)", m);
    if ((double)N * (2.0 * m + 1.0) * (2.0 * m + 1.0) >= 2147483647.0)
        return fail2(INFFT_EINVAL, "N (2m+1)^2 must be < 2^31 (N = %lld, m = %d)", (long long)N, m);
    infft2d_plan_s* p = new infft2d_plan_s();
    cudaGetDevice(&p->device);
    p->M1 = M1; p->M2 = M2; p->Ms1 = Ms1; p->Ms2 = Ms2; p->N = N; p->P = Ms1 * Ms2;
    p->m = m; p->kernel = kernel; p->sigma = sigma; p->tau = tau; p->log1 = l1; p->log2 = l2;
    p->nnz_cap = N * (2 * (int64_t)m + 1) * (2 * (int64_t)m + 1);
    Carver2 c;
    layout2(p, c);
    cudaError_t e = cudaMalloc(&p->arena, c.off);
    if (e == cudaSuccess) {
        c.base = (char*)p->arena;
        c.off = 0;
        layout2(p, c);
        e = cudaMemset(p->counters, 0, C2_N * sizeof(int32_t));
    }
    if (e != cudaSuccess) {
        if (p->arena) cudaFree(p->arena);
        delete p;
        return cuda_fail2(e, "allocate plan buffers");
    }
    *out = p;
    return INFFT_OK;
}

infft_status infft2d_set_nodes(infft2d_plan_t p, const double* x, infft_stream_t stream) {
    if (!p) return fail2(INFFT_EINVAL, "plan is NULL");
    if (!x) return fail2(INFFT_EINVAL, "x is NULL");
    DeviceGuard2 g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    p->nodes_set = 0;
    p->precomputed = 0;
    cudaError_t e;
    if (on_device2(x)) {
        e = cudaMemcpyAsync(p->x, x, p->N * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    } else {
        const int64_t j = first_bad_coordinate(x, 2 * p->N);
        if (j >= 0)
            return fail2(INFFT_EINVAL, "node coordinate x[%lld] = %.17g is not in [-1/2, 1/2)", (long long)j, x[j]);
        e = cudaMemcpyAsync(p->x, x, p->N * sizeof(double2), cudaMemcpyHostToDevice, s);
    }
    if (e != cudaSuccess) return cuda_fail2(e, "copy nodes");
    if ((e = run_pattern2(p, s)) != cudaSuccess) return cuda_fail2(e, "pattern");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail2(e, "synchronize");
    int32_t cnt[C2_N];
    if ((e = cudaMemcpy(cnt, p->counters, sizeof cnt, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail2(e, "read counters");
    if (cnt[C2_BAD] > 0) return fail2(INFFT_EINVAL, "%d nodes are not finite or not in [-1/2, 1/2)^2", cnt[C2_BAD]);
    int32_t nnz = 0;
    if ((e = cudaMemcpy(&nnz, p->col_off + p->P, sizeof nnz, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail2(e, "read nnz");
    p->nnz = nnz;
    p->max_column = cnt[C2_MAX_COLUMN];
    p->nodes_set = 1;
    return INFFT_OK;
}

infft_status infft2d_precompute(infft2d_plan_t p, infft_stream_t stream) {
    if (!p) return fail2(INFFT_EINVAL, "plan is NULL");
    if (!p->nodes_set) return fail2(INFFT_ENOTREADY, "infft2d_precompute before infft2d_set_nodes");
    DeviceGuard2 g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = run_precompute2(p, s);
    // the large-column scratch (gigabytes for clustered nodes) is not kept between precomputes
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        if (p->scratch) cudaFree(p->scratch);
        if (p->gscratch) cudaFree(p->gscratch);
        p->scratch = p->gscratch = nullptr;
        p->scratch_doubles = p->gscratch_doubles = 0;
    }
    if (e != cudaSuccess) return cuda_fail2(e, "precompute");
    p->precomputed = 1;
    return INFFT_OK;
}

infft_status infft2d_apply(infft2d_plan_t p, const float* f, float* fhat, infft_stream_t stream) {
    return apply2_impl<float>(p, f, fhat, stream);
}

infft_status infft2d_apply_z(infft2d_plan_t p, const double* f, double* fhat, infft_stream_t stream) {
    return apply2_impl<double>(p, f, fhat, stream);
}

infft_status infft2d_get_info(infft2d_plan_t p, infft2d_info* info) {
    if (!p || !info) return fail2(INFFT_EINVAL, "plan and info must not be NULL");
    DeviceGuard2 g(p->device);
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    if (e != cudaSuccess) return cuda_fail2(e, "synchronize");
    int32_t cnt[C2_N];
    if ((e = cudaMemcpy(cnt, p->counters, sizeof cnt, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail2(e, "read counters");
    std::memset(info, 0, sizeof *info);
    info->M1 = p->M1; info->M2 = p->M2; info->M_sigma1 = p->Ms1; info->M_sigma2 = p->Ms2; info->N = p->N;
    info->m = p->m; info->kernel = p->kernel; info->sigma = p->sigma; info->tau = p->tau;
    info->nodes_set = p->nodes_set;
    info->precomputed = p->precomputed;
    info->bad_nodes = cnt[C2_BAD];
    if (p->nodes_set) {
        info->nnz = p->nnz;
        info->max_column = cnt[C2_MAX_COLUMN];
        info->empty_columns = cnt[C2_EMPTY];
    }
    if (p->precomputed) {
        info->fallback_columns = cnt[C2_FALLBACK];
        info->unsupported_columns = cnt[C2_UNSUPPORTED];
        info->large_columns = cnt[C2_LIST0 + 3] + cnt[C2_LIST0 + 4];
        info->wide_columns = cnt[C2_WIDE];
        info->indexed_columns = cnt[C2_INDEXED];
        std::string buf(p->P * sizeof(double), '\0');
        if ((e = cudaMemcpy(&buf[0], p->J, p->P * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail2(e, "read objective");
        const double* J = (const double*)buf.data();
        double sum = 0.0;
        for (int64_t i = 0; i < p->P; ++i) sum += J[i];
        info->objective = sum;
    }
    return INFFT_OK;
}

infft_status infft2d_copy_plan_data(infft2d_plan_t p, int32_t* col_offset, int32_t* col_node, double* weights,
                                    double* objective) {
    if (!p) return fail2(INFFT_EINVAL, "plan is NULL");
    if (!p->nodes_set) return fail2(INFFT_ENOTREADY, "no nodes set");
    if ((weights || objective) && !p->precomputed) return fail2(INFFT_ENOTREADY, "not precomputed");
    DeviceGuard2 g(p->device);
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    if (e == cudaSuccess && col_offset) e = cudaMemcpy(col_offset, p->col_off, (p->P + 1) * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && col_node) e = cudaMemcpy(col_node, p->col_node, (size_t)p->nnz * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && weights) e = cudaMemcpy(weights, p->w64, (size_t)p->nnz * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && objective) e = cudaMemcpy(objective, p->J, p->P * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail2(e, "copy plan data");
    return INFFT_OK;
}

infft_status infft2d_plan_destroy(infft2d_plan_t p) {
    if (!p) return INFFT_OK;
    {
        DeviceGuard2 g(p->device);
        cudaDeviceSynchronize();
        if (p->scratch) cudaFree(p->scratch);
        if (p->gscratch) cudaFree(p->gscratch);
        if (p->gdesc) cudaFree(p->gdesc);
        if (p->gprefix) cudaFree(p->gprefix);
        if (p->arena) cudaFree(p->arena);
    }
    delete p;
    return INFFT_OK;
}

}  // extern "C"
