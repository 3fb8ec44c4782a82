// Internal plan object and the launch functions each translation unit provides.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/infft.h"
#include "common.cuh"

// device counters (int32), read back by infft_get_info
enum {
    CNT_BAD_NODES = 0,
    CNT_FALLBACK = 1,
    CNT_UNSUPPORTED = 2,
    CNT_MAX_COLUMN = 3,
    CNT_EMPTY = 4,
    CNT_LIST_A = 5,        // columns queued for the warp solver
    CNT_BIG_SEGMENTS = 6,  // buckets queued for the large-bucket fix-up of the pattern sort
    CNT_BIG_LIST = 7,      // columns queued for the CTA solver
    CNT_TILES_MID = 8,     // tiles routed to the 25-node thread tier
    CNT_TILES_BIG = 9,     // tiles routed to the 33-node thread tier
    CNT_GRAD_FAIL = 10,    // columns the node gradient could not factor (or too large)
    CNT_HUGE_LIST = 11,    // batch members: columns above 224 nodes solved by the batch's blocked solver
    CNT_TILES_48 = 12,     // tiles routed to the 48-node group tier
    CNT_TILES_64 = 13,     // tiles routed to the 64-node group tier
    CNT_N = 14
};

// largest column handled by the thread, warp and CTA solver tiers
constexpr int LSQ_THREAD_NMAX1 = 17;
constexpr int LSQ_THREAD_NMAX2 = 25;
constexpr int LSQ_THREAD_NMAX3 = 33;
constexpr int LSQ_WARP2_NMAX = 64;
constexpr int LSQ_GROUP_G2 = 4;      // lanes per column in the <= 25 tier
constexpr int LSQ_GROUP_G3 = 8;      // lanes per column in the <= 33 tier
constexpr int LSQ_GROUP_NMAX4 = 48;  // tiles of columns up to 48 nodes: 16 lanes per column, sub-tiles of 16
constexpr int LSQ_GROUP_G4 = 16;
constexpr int LSQ_GROUP_TC4 = 16;
constexpr int LSQ_GROUP_G5 = 32;     // up to 64 nodes (LSQ_WARP2_NMAX): a warp per column, sub-tiles of 8
constexpr int LSQ_GROUP_TC5 = 8;
constexpr int LSQ_CTA_NMAX = 224;
// largest |I(x_j)| = 2m + 1 of the underdetermined case
constexpr int UNDER_NMAX = 17;

// Columns whose ||b_l||_1 exceeds this are spread and interpolated in float-float on the
// fp32 pipe (weights as fp32 pairs hi + lo, exact products, compensated sums; ffsum.cuh):
// their terms cancel, and fp32 rounding of O(||b_l||_1 |f|) terms would dominate the result.
constexpr double WIDE_COLUMN_L1 = 32.0;

struct ProfileRec {
    const char* name;
    cudaEvent_t start, stop;
};

struct infft_plan_s {
    int device = 0;
    int64_t M = 0, N = 0, Ms = 0;
    int m = 0, kernel = INFFT_KERNEL_FULL, ansatz = INFFT_ANSATZ_OVERDETERMINED;
    double sigma = 2.0, tau = 1e-12;
    int logMs = 0;
    int64_t nnz_cap = 0;

    // pattern (a1)
    double* x = nullptr;        // nodes, caller order (N)
    double* xs = nullptr;       // nodes, sorted (N)
    double2* phase = nullptr;   // N: (sin, cos)(pi M x) of the sorted nodes
    uint32_t* skey = nullptr;   // N: key of each sorted node (2 cell + (u not an integer))
    int32_t* perm = nullptr;    // N: sorted position -> caller index
    int32_t* bucket = nullptr;  // 2 Ms + 1: key counts, then their exclusive prefix (bucket offsets)
    int32_t* cursor = nullptr;  // 2 Ms: scatter cursors of the counting sort
    int32_t* seg_list = nullptr;// buckets larger than one thread orders
    int32_t* sort_tmp = nullptr;// N: scratch of the large-bucket fix-up
    int32_t* col_start = nullptr;   // Ms
    int32_t* col_count = nullptr;   // Ms
    int32_t* col_off = nullptr;     // Ms + 1
    int32_t* list_a = nullptr;      // Ms (columns for the 32-row warp solver)
    int32_t* tiles_mid = nullptr;   // Ms/32 + 1 (tiles for the 25-node thread tier)
    int32_t* tiles_big = nullptr;   // Ms/32 + 1 (tiles for the 33-node thread tier)
    int32_t* tiles_48 = nullptr;    // Ms/32 + 1 (tiles for the 48-node group tier)
    int32_t* tiles_64 = nullptr;    // Ms/32 + 1 (tiles for the 64-node group tier)
    int32_t* big_list = nullptr;    // Ms (columns for the CTA solver)
    int32_t* scan_sums = nullptr;   // per-block partial sums of the scans
    int32_t* counters = nullptr;    // CNT_N

    // B_opt (a2)
    double* w64 = nullptr;      // nnz_cap
    float* w32 = nullptr;       // nnz_cap
    double* J = nullptr;        // Ms (overdetermined), N (underdetermined, caller order)
    uint8_t* wide = nullptr;    // Ms: 1 if column l spreads in float-float in the fp32 applies
    float* wlo = nullptr;       // nnz_cap: fp32(w64 - w32), the low parts of the float-float weights
    double* gterm = nullptr;    // nnz_cap: per (column, node) terms of the node gradient

    // underdetermined case (Sec. 3.2.1)
    void* under_step = nullptr; // N double2: exp(2 pi i x_h) of the sorted nodes
    void* under_part = nullptr; // chunks * M double2: partial node moments
    void* under_mom = nullptr;  // M double2: node moments mu_n, n = 0 .. M-1
    void* under_S = nullptr;    // (2m+1) * Ms double2: S(l' + d, l'), d = 0 .. 2m

    // apply buffers (a3-a5)
    void* grid = nullptr;       // Ms double2 (also used as float2)
    void* work = nullptr;       // Ms double2 (FFT intermediate)
    void* stage_in = nullptr;   // max(N, M) double2: host-input staging
    void* stage_out = nullptr;  // max(N, M) double2: host-output staging

    void* arena = nullptr;      // the one device allocation holding the buffers above (owned)
    // M_sigma not a power of two (sigma = 2, M <= 8192): the plan is a batch of one problem,
    // whose FFT is the chirp convolution (batch.cu); only set_nodes, precompute, the fp32 apply,
    // get_info and copy_plan_data are available (owned)
    infft_batch_t chirp = nullptr;
    bool batch_member = false;  // buffers carved from a batch; big columns go to the batch's solver
    int nodes_set = 0, precomputed = 0;
    int apply_clean = 0;        // 0 after set_nodes / precompute until the next apply has been launched
    int apply_cfg = -1;         // tile shape of the fused apply (-1: the default rule)
    int lay_cfg = -1;           // tile shape the apply layout below holds (-1: none, or stale)
    int sms = 0;                // multiprocessors of the plan's device

    // apply layout of the fused apply (apply.cu): per tile a header, per column a descriptor,
    // the weights and node-window lists tile by tile
    int4* lay_hdr = nullptr;          // max tiles
    uint2* lay_cdesc = nullptr;       // Ms
    float* lay_w = nullptr;           // apply2_weight_capacity
    int32_t* lay_list = nullptr;      // apply2_list_capacity: caller indices
    int32_t* lay_list_sorted = nullptr;   // the same windows as sorted positions
    int32_t* lay_tmp = nullptr;       // 5 max tiles: block lengths, direct flags, block starts
    cudaStream_t last_stream = nullptr;

    bool profiling = false;
    std::vector<ProfileRec> prof;
};

typedef infft_plan_s Plan;

// Lays a plan's device buffers out in one arena.  With base == nullptr it only
// measures (off grows by the bytes needed); every buffer starts on a 256-byte
// boundary and has 16 bytes of slack behind it (vector loads may overrun).
struct Carver {
    char* base = nullptr;
    size_t off = 0;
    template <typename X> void take(X*& ptr, size_t count) {
        off = (off + 255) & ~(size_t)255;
        ptr = base ? (X*)(base + off) : nullptr;
        off += count * sizeof(X) + 16;
    }
};

// Buffers of plan p (sizes from p->M, N, Ms, m, ansatz).  A batch member gets
// neither x (it points into the batch's node array) nor the buffers of the
// single-problem applies, staging and node gradient.
void plan_layout(Plan* p, Carver& c, bool batch_member);

// Host check of node coordinates: the index of the first one outside [-1/2, 1/2) or not finite
// (NaN fails both comparisons), or -1.  A branch-free count runs first, which the compiler
// vectorises (a loop that exits at the first bad value does not vectorise).
int64_t first_bad_coordinate(const double* x, int64_t n);

// Records a failure for infft_last_error() and returns st.
infft_status set_error(infft_status st, const char* fmt, ...);
// Adds to the library's launch counter (infft_launch_count) for launches made without a plan.
void count_launches(int n);

// Launch bookkeeping: counts launches and, when profiling, brackets each launch
// with an event pair on its stream.
void launch_begin(Plan* p, const char* name, cudaStream_t s);
void launch_end(Plan* p, cudaStream_t s);

// pattern.cu
cudaError_t run_pattern(Plan* p, cudaStream_t s);
// pattern.cu: the pattern of every problem of a batch in one launch (one CTA per problem,
// problems in `order`, largest first); PatternArgs on the device
struct PatternArgs {
    const double* x;
    double* xs;
    double2* phase;
    uint32_t* skey;
    int32_t* perm;
    int32_t* bucket;
    int32_t* cursor;
    int32_t* seg_list;
    int32_t* sort_tmp;
    int32_t* col_start;
    int32_t* col_count;
    int32_t* col_off;
    int32_t* counters;
    int N, Ms, m;
    double M;
};
cudaError_t run_pattern_batch(const PatternArgs* probs, const int32_t* order, int P, int sms, cudaStream_t s);
// pattern.cu: fills the node-phase table on the current device (once; synchronous, so it is
// called when a plan or batch is created, not inside a stream capture)
cudaError_t phase_table_init();
cudaError_t run_exclusive_scan(Plan* p, const int32_t* in, int32_t* out, int n, cudaStream_t s);
// lsq.cu
cudaError_t run_precompute(Plan* p, cudaStream_t s);
// lsq.cu: the blocked solver over the big lists (columns above 64 nodes) of P batch members;
// job_off: P + 1 ints of device scratch; scratch: huge_scratch_doubles(slots, nmax) doubles,
// nmax <= HUGE_NMAX the largest column it solves (larger ones: b_l = 0, counted unsupported)
constexpr int HUGE_NMAX = 1024;
size_t huge_problem_bytes();                                   // size of one device descriptor
void huge_problems_fill(Plan* const* plans, int P, void* host); // P descriptors into host memory
size_t huge_scratch_doubles(int slots, int nmax);
// order: one int per possible job (sum of the problems' M_sigma); work: nmax + 8 ints
cudaError_t run_precompute_huge(const void* probs, int P, int32_t* job_off, int32_t* order, int32_t* work,
                                double* scratch, int slots, int nmax, cudaStream_t s);
// lsq.cu: the solver tiers of every problem of a batch, one launch per tier.  probs: P device
// descriptors (tier_args of each member, tier_args_bytes() each); tile_off: P + 1 device
// prefix of the problems' 32-column tiles; off_work: 3 (P + 1) ints of device scratch.  Columns
// above 64 nodes stay in the members' big lists (run_precompute_huge).
size_t tier_args_bytes();
void tier_args_fill(Plan* const* plans, int P, void* host);
cudaError_t run_precompute_batch(const void* probs, int P, const int32_t* tile_off, int total_tiles,
                                 int32_t* off_work, int sms, cudaStream_t s);
// under.cu: the underdetermined case; under_moment_chunks = partial-sum blocks of the node moments
cudaError_t run_precompute_under(Plan* p, cudaStream_t s);
int under_moment_chunks(int64_t N);
// spread.cu: g = B_opt^* f onto p->grid (T = float or double, complex layout)
template <typename T> cudaError_t run_spread(Plan* p, const void* f, cudaStream_t s);
// spread.cu: f = B_opt g from p->grid, f in caller node order
template <typename T> cudaError_t run_interp(Plan* p, void* f, cudaStream_t s);
// fft.cu: fhat = D^* F^* grid (pruned to the M central frequencies)
template <typename T> cudaError_t run_fft_adjoint(Plan* p, void* fhat, cudaStream_t s);
// spread.cu / fft.cu: the fp32 apply of K data vectors (f: K x N, grid and work: K x M_sigma,
// fhat: K x M); the FFT requires M_sigma > 2048
cudaError_t run_spread_many(Plan* p, const void* f, void* grid, int K, cudaStream_t s);
cudaError_t run_fft_adjoint_many(Plan* p, const void* grid, void* work, void* fhat, int K, cudaStream_t s);
// apply.cu: the fp32 apply in two launches (spreading fused with FFT pass A, then pass B with D);
// sorted: f is given in the plan's sorted node order.  Tile shapes ("configs") are numbered
// 0 .. apply2_config_count() - 1; valid ones depend on M_sigma.
int apply2_config_count();
bool apply2_config_valid(const Plan* p, int id);
int apply2_default_config(const Plan* p);
// K data vectors (f: K x N, fhat: K x M) with pass A's output in Y (K x M_sigma; nullptr: the
// plan's work buffer, K = 1)
cudaError_t run_apply2(Plan* p, const float2* f, bool sorted, float2* fhat, cudaStream_t s, int K = 1,
                       float2* Y = nullptr);
int64_t apply2_max_tiles(const Plan* p);
int64_t apply2_list_capacity(const Plan* p);
int64_t apply2_weight_capacity(const Plan* p);
void apply2_config_shape(int id, int* log1, int* C);
// apply.cu: out[i] = f[perm[i]] (sort) and out[perm[i]] = f[i] (unsort), complex64
cudaError_t run_sort_values(Plan* p, const float2* f, float2* out, cudaStream_t s);
cudaError_t run_unsort_values(Plan* p, const float2* f, float2* out, cudaStream_t s);
// fft.cu: pass B of the four-step FFT alone (rows of length 2^log2), D fused, pruned output
cudaError_t fft_passB_r8(const float2* work, float2* fhat, int log1, int log2, int M, int sym, cudaStream_t s,
                         Plan* p, int K = 1);
// fft.cu: grid = F D fhat
template <typename T> cudaError_t run_fft_forward(Plan* p, const void* fhat, cudaStream_t s);
// fft.cu: out_p = scale * sum_{k=-Ms/2}^{Ms/2-1} in[k + Ms/2] exp(2 pi i k (p - Ms/2)/Ms), fp64, all bins
cudaError_t run_fft_full_forward_z(Plan* p, const void* in, void* out, double scale, cudaStream_t s);
// fft.cu: out_p = sum_{k=-M/2}^{M/2-1} in[k + M/2] exp(2 pi i k (p - Ms/2)/Ms), fp64, all Ms bins
cudaError_t run_fft_forward_band_z(Plan* p, const void* in, void* out, cudaStream_t s);
// grad.cu: gx = dL/dx (caller order) for f (complex64, device) and w = dL/dfhat (complex64, device)
cudaError_t run_grad_nodes(Plan* p, const void* f, const void* w, double* gx, cudaStream_t s);
// fft.cu: the fp32 2-D transform of the tensor-product plan: grid g (2^log1 x 2^log2 complex64,
// row-major) -> fhat (M1 x M2, k1-major, (-1)^(k1+k2) d_k applied); Y holds 2^log1 x M2 complex64.
// Supported for 2^log_t in [64, 2048] with M2 a multiple of the column pass's CTA width.
bool fft2d_r8_supported(int log1, int log2, int M2);
cudaError_t fft2d_adjoint_r8(const float2* g, float2* Y, float2* fhat, int log1, int log2, int M1, int M2, int sym,
                             cudaStream_t s);
// refine.cu: out = A fhat by the direct fp64 sum over the plan's nodes (caller order), or
// resid - A fhat when resid is given (N complex128 each); y += d (n complex128)
cudaError_t run_ndft_z(Plan* p, const void* fhat, const void* resid, void* out, cudaStream_t s);
// refine.cu: the same with the windowed NFFT (Kaiser-Bessel, Sec. 2.1) when nfft_kb_supported(p);
// scratch: p->grid, p->work and `coef` (M complex128)
bool nfft_kb_supported(const Plan* p);
cudaError_t run_nfft_kb_z(Plan* p, const void* fhat, const void* resid, void* out, void* coef, cudaStream_t s);
cudaError_t run_axpy_z(Plan* p, void* y, const void* d, int n, cudaStream_t s);
