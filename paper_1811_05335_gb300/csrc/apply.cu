// The fp32 modified adjoint NFFT fhat = D^* F^* B_opt^* f (eq:approx_ansatz2) in two
// launches: the spreading g = B_opt^* f fused with the first pass of the four-step FFT,
// then the second pass with the deconvolution D^* and the pruning to the M kept
// frequencies (k_fftB_r8).
//
// Four-step split M_sigma = N1 * N2 with grid index p = N2 p1 + p2 (p = l + M_sigma/2):
// pass A needs, for a fixed p2, the grid values at all N1 indices p1.  A CTA of the fused
// kernel ("tile") therefore owns C consecutive p2 values and spreads the N1 runs of C
// consecutive grid points {N2 p1 + p2_0 .. N2 p1 + p2_0 + C - 1}.  Grid point l couples to
// the sorted nodes of a contiguous (wrapping) range, so each run's nodes form one window of
// sorted nodes.
//
// Apply layout.  After the precompute, a preparation pass lays each tile's data out
// contiguously: its weights (column by column, in the tile's column order, one unused slot
// after each column so that a warp's columns start on different shared-memory banks), the caller
// indices (and the sorted positions) of its runs' node windows, and one 8-byte descriptor
// per column (weight offset and count, offset of its first node in the window list, the
// float-float flag).  A tile header gives the block positions and lengths; tiles that
// exceed the staging buffers (clustered nodes) are marked and read the plan's column arrays
// directly.  The fused kernel then only streams contiguous blocks with 16-byte
// asynchronous copies, gathers the data vector through its node list, sums each grid point's
// column from shared memory, runs the C length-N1 transforms in registers, multiplies by
// w^{p2 k1} and stores Y[k1 N2 + p2] (1 MiB at M_sigma = 2^17, which stays in L2 for pass B).
//
// Plan-owned data (header, descriptors, weights, node lists) is read before the kernel waits
// on its predecessor in the stream (programmatic dependent launch): when that predecessor is
// the previous apply's pass B, the copies overlap it.  Only the data vector f is read, and Y
// written, after the wait.  The launch that follows set_nodes, precompute or a change of the
// tile shape is an ordinary one, so those copies never overlap the kernels that wrote the
// data.
#include "plan.h"
#include "fft_r8.cuh"
#include "ffsum.cuh"

namespace {

constexpr int A1_WMAX = 12288;                        // staged weights per tile (48 KB)
constexpr int A1_UMAX = 4096;                         // staged node values per tile (32 KB)
constexpr int A1_NCOL_MAX = 512;

struct A1Args {
    const float2* f;          // N data values, caller order (sorted order when SORTED)
    const int4* hdr;          // per tile: weight block start, length; node block start, length (-1: direct)
    const uint2* cdesc;       // per column of each tile (tile-major): woff | n << 16, uoff | wide << 31
    const float* aw;          // weights, tile-major
    const int32_t* alist;     // node window lists, tile-major: caller indices (sorted positions when SORTED)
    // the plan's column arrays, for tiles read directly
    const float* w32;         // B_opt weights, column-major
    const float* wlo;         // low parts w64 - fp32(w64) (float-float for wide columns)
    const uint8_t* wide;      // M_sigma: 1 where ||b_l||_1 is large and terms cancel
    const int32_t* perm;      // sorted position -> caller index
    const int32_t* col_start; // M_sigma: first sorted node of I(l)
    const int32_t* col_off;   // M_sigma + 1: weight offset of column l
    float2* Y;                // M_sigma: Y[k1 N2 + p2]
    int N;
    int log2;                 // N2 = 2^log2
};

// g_l of one column by direct global loads (tiles that do not fit the staging buffers)
template <bool SORTED>
INFFT_D float2 column_direct(const A1Args& a, int p) {
    const int off = a.col_off[p], n = a.col_off[p + 1] - off;
    int q = a.col_start[p];
    if (!a.wide[p]) {
        float re = 0.f, im = 0.f;
        for (int i = 0; i < n; ++i) {
            const float wi = a.w32[off + i];
            const float2 v = a.f[SORTED ? q : a.perm[q]];
            re = fmaf(wi, v.x, re);
            im = fmaf(wi, v.y, im);
            if (++q == a.N) q = 0;
        }
        return make_float2(re, im);
    }
    FFSum s;
    for (int i = 0; i < n; ++i) {
        s.add(a.w32[off + i], a.wlo[off + i], a.f[SORTED ? q : a.perm[q]]);
        if (++q == a.N) q = 0;
    }
    return s.value();
}

template <int LOG1, int C>
struct A1Layout {
    static constexpr int N1 = 1 << LOG1, NCOL = N1 * C;
    static constexpr int W_BYTES = A1_WMAX * 4, U_BYTES = A1_UMAX * 8, L_BYTES = A1_UMAX * 4;
    static constexpr int BYTES = W_BYTES + U_BYTES + L_BYTES + NCOL * 8 + N1 * 8;
};

// The fused spreading and pass A of tile b (blockIdx.x): columns j = r C + c (run r < N1,
// c < C) at grid point p = N2 r + C b + c.  Thread t sums columns t, t + 256, ...; the
// first NCOL / 8 threads then run the C length-N1 transforms (8 values each; thread t:
// transform t mod C, slot t / C).
template <int LOG1, int C, bool SORTED>
__global__ void __launch_bounds__(256, 2)
k_apply_spread_fftA(A1Args a) {
    using L = A1Layout<LOG1, C>;
    constexpr int N1 = L::N1, NCOL = L::NCOL, T1 = N1 / 8, RS = N1 + N1 / 8;
    constexpr int A1_THREADS = 256, CPT = NCOL / 256;
    static_assert(NCOL <= A1_NCOL_MAX, "tile shape");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* ws = (float*)smem_raw;                                                   // weights
    float2* fu = (float2*)(smem_raw + L::W_BYTES);                                  // node values
    int32_t* sl = (int32_t*)(smem_raw + L::W_BYTES + L::U_BYTES);                   // node list
    uint2* cd = (uint2*)(smem_raw + L::W_BYTES + L::U_BYTES + L::L_BYTES);          // column descriptors
    float2* tw = (float2*)(smem_raw + L::W_BYTES + L::U_BYTES + L::L_BYTES + NCOL * 8);   // N1 twiddles
    const int tid = threadIdx.x, log2 = a.log2, b = blockIdx.x;
    // data vector blockIdx.y of several (apply_many): f at y N, Y at y M_sigma
    a.f += (size_t)blockIdx.y * a.N;
    a.Y += (size_t)blockIdx.y * ((size_t)N1 << log2);

    // ---- plan-owned data (before the wait on the previous kernel) ----
    r8_twiddles<N1>(tw, tid, A1_THREADS);
    const int4 h = a.hdr[b];
    const bool staged = h.y >= 0;
    if (staged) {
        const uint4* src = (const uint4*)(a.cdesc + (size_t)b * NCOL);
        for (int k = tid; k < NCOL / 2; k += A1_THREADS) cp_async16(cd + 2 * k, src + k);
        for (int k = tid; k < h.y / 4; k += A1_THREADS) cp_async16(ws + 4 * k, a.aw + h.x + 4 * k);
        for (int k = tid; k < h.w / 4; k += A1_THREADS) cp_async16(sl + 4 * k, a.alist + h.z + 4 * k);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }

    // ---- the data vector (after the wait) ----
    griddep_wait();
    griddep_launch();
    float2 val[CPT];
    if (staged) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        for (int q = tid; q < h.w / 4; q += A1_THREADS) {
            const int4 ix = ((const int4*)sl)[q];
            cp_async8(fu + 4 * q, a.f + ix.x);
            cp_async8(fu + 4 * q + 1, a.f + ix.y);
            cp_async8(fu + 4 * q + 2, a.f + ix.z);
            cp_async8(fu + 4 * q + 3, a.f + ix.w);
        }
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const uint2 d = cd[tid + k * A1_THREADS];
            const int woff = (int)(d.x & 0xffffu), n = (int)(d.x >> 16), uoff = (int)(d.y & 0x7fffffffu);
            const float* wc = ws + woff;
            const float2* fc = fu + uoff;
            if (d.y >> 31) {
                const int j = tid + k * A1_THREADS, r = j / C, c = j - r * C;
                const int p = (r << log2) + C * b + c;
                const int off = a.col_off[p];
                FFSum s;
                for (int i = 0; i < n; ++i) s.add(wc[i], a.wlo[off + i], fc[i]);
                val[k] = s.value();
                continue;
            }
            float re = 0.f, im = 0.f, re2 = 0.f, im2 = 0.f;
            int i = 0;
            for (; i + 4 <= n; i += 4) {
                const float w0 = wc[i], w1 = wc[i + 1], w2 = wc[i + 2], w3 = wc[i + 3];
                const float2 v0 = fc[i], v1 = fc[i + 1], v2 = fc[i + 2], v3 = fc[i + 3];
                re = fmaf(w0, v0.x, re);
                im = fmaf(w0, v0.y, im);
                re2 = fmaf(w1, v1.x, re2);
                im2 = fmaf(w1, v1.y, im2);
                re = fmaf(w2, v2.x, re);
                im = fmaf(w2, v2.y, im);
                re2 = fmaf(w3, v3.x, re2);
                im2 = fmaf(w3, v3.y, im2);
            }
            for (; i < n; ++i) {
                const float wi = wc[i];
                const float2 v = fc[i];
                re = fmaf(wi, v.x, re);
                im = fmaf(wi, v.y, im);
            }
            val[k] = make_float2(re + re2, im + im2);
        }
    } else {
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const int j = tid + k * A1_THREADS, r = j / C, c = j - r * C;
            val[k] = column_direct<SORTED>(a, (r << log2) + C * b + c);
        }
    }
    __syncthreads();   // ws is reused below
    // transform c's input, element p1 = r: gin[c N1 + r]
    float2* gin = (float2*)smem_raw;
    float2* bufs = gin + NCOL;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const int j = tid + k * A1_THREADS, r = j / C, c = j - r * C;
        gin[c * N1 + r] = val[k];
    }
    __syncthreads();
    constexpr int FT = NCOL / 8;   // threads of the C transforms
    if (tid >= FT) return;
    const int c = tid % C, jj = tid / C;
    float2 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = gin[c * N1 + jj + r * T1];
    float2* bufA = bufs + 2 * c * RS;
    fft_r8<LOG1, -1, NamedSync<1, FT>>(v, bufA, bufA + RS, tw, jj);
    // w^{p2 k1} for the bins k1 = jj + b N1/8 + r N1/R of this thread: three exact
    // evaluations and products (at most 8 roundings)
    const int p2 = C * b + c;
    const int Ms = N1 << log2;
    constexpr int R = (LOG1 % 3) ? (1 << (LOG1 % 3)) : 8;
    const float2 wj = expm2pi_frac(p2 * jj, Ms), wb = expm2pi_frac(p2 * (N1 / 8), Ms),
                 wr = expm2pi_frac(p2 * (N1 / R), Ms);
    float2 rowb = wj;
#pragma unroll
    for (int bb = 0; bb < 8 / R; ++bb) {
        float2 w = rowb;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int s = bb * R + r;
            a.Y[(r8_bin<LOG1>(jj, s) << log2) + p2] = cmul(v[s], w);
            w = cmul(w, wr);
        }
        rowb = cmul(rowb, wb);
    }
}

// ---- the apply layout -------------------------------------------------------------

// Window of the run starting at grid point p0 (C columns): the sorted nodes [S, S + U)
// (mod N) covering them, and whether every column's range lies inside it.
struct RunWindow {
    int S, U, ok;
};

INFFT_D RunWindow run_window(const int32_t* col_off, const int32_t* col_start, int N, int p0, int C) {
    RunWindow w;
    w.S = col_start[p0];
    const int last = p0 + C - 1;
    int U = col_start[last] + (col_off[last + 1] - col_off[last]) - w.S;
    if (U < 0) U += N;
    int ok = U <= N;
    for (int c = 0; c < C; ++c) {
        const int n = col_off[p0 + c + 1] - col_off[p0 + c];
        int r0 = col_start[p0 + c] - w.S;
        if (r0 < 0) r0 += N;
        ok &= (n == 0) | (r0 + n <= U);
    }
    w.U = U;
    w.ok = ok;
    return w;
}

INFFT_D int pad4(int v) { return (v + 3) & ~3; }

// sum over the block (blockDim.x threads, a multiple of 32, at most 1024); every thread
// gets the total
INFFT_D int block_sum(int v, int* red) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < nw; ++w) t += red[w];
    return t;
}

// Pass 1: tile b's block lengths (weights and node list, padded to 16 bytes), or 0 for a tile
// whose data does not fit the staging buffers or whose windows are not contiguous.
__global__ void k_layout_count(const int32_t* __restrict__ col_off, const int32_t* __restrict__ col_start, int N,
                               int log1, int log2, int C, int32_t* __restrict__ wlen, int32_t* __restrict__ ulen,
                               int32_t* __restrict__ direct) {
    __shared__ int red[32];
    const int b = blockIdx.x, N1 = 1 << log1;
    int w = 0, u = 0, bad = 0;
    for (int r = threadIdx.x; r < N1; r += blockDim.x) {
        const int p0 = (r << log2) + C * b;
        w += col_off[p0 + C] - col_off[p0] + C;   // + one skew slot per column
        const RunWindow rw = run_window(col_off, col_start, N, p0, C);
        u += rw.U;
        bad += !rw.ok;
    }
    w = block_sum(w, red);
    u = block_sum(u, red);
    bad = block_sum(bad, red);
    if (threadIdx.x == 0) {
        const bool fits = bad == 0 && pad4(w) <= A1_WMAX && pad4(u) <= A1_UMAX;
        wlen[b] = fits ? pad4(w) : 0;
        ulen[b] = fits ? pad4(u) : 0;
        direct[b] = !fits;
    }
}

// Pass 2 (wstart, ustart: exclusive prefix sums of the lengths): header, weights, node lists
// and column descriptors of tile b.  The tile's column offsets and starts are staged in
// shared memory once; the runs' offsets within the tile's blocks come from a block scan.
__global__ void __launch_bounds__(1024)
k_layout_fill(const int32_t* __restrict__ col_off, const int32_t* __restrict__ col_start,
              const float* __restrict__ w32, const uint8_t* __restrict__ wide, const int32_t* __restrict__ perm,
              int N, int log1, int log2, int C, const int32_t* __restrict__ wstart, const int32_t* __restrict__ ustart,
              const int32_t* __restrict__ wlen, const int32_t* __restrict__ ulen, const int32_t* __restrict__ direct,
              int64_t wcap, int64_t lcap, int4* __restrict__ hdr, uint2* __restrict__ cdesc, float* __restrict__ aw,
              int32_t* __restrict__ alist, int32_t* __restrict__ alist_sorted) {
    __shared__ int s_off[A1_NCOL_MAX + 256];   // N1 (C + 1) column offsets (N1 <= 256, N1 C <= 512)
    __shared__ int s_st[A1_NCOL_MAX];          // N1 C column starts
    __shared__ int wrun[257], urun[257], rS[256], red[64];
    const int b = blockIdx.x, N1 = 1 << log1, NCOL = N1 * C, tid = threadIdx.x;
    // a tile whose blocks would end beyond the buffers' capacities is read directly (cannot
    // happen: the capacities bound the sums of all tiles' blocks; a guard all the same)
    if (direct[b] || (int64_t)wstart[b] + wlen[b] > wcap || (int64_t)ustart[b] + ulen[b] > lcap) {
        if (tid == 0) hdr[b] = make_int4(0, -1, 0, -1);
        return;
    }
    for (int i = tid; i < N1 * (C + 1); i += blockDim.x) {
        const int r = i / (C + 1), c = i - r * (C + 1);
        s_off[i] = col_off[(r << log2) + C * b + c];
    }
    for (int i = tid; i < NCOL; i += blockDim.x) {
        const int r = i / C, c = i - r * C;
        s_st[i] = col_start[(r << log2) + C * b + c];
    }
    __syncthreads();
    // per run (thread r): weights incl. one skew slot per column, window start and length
    int W = 0, U = 0;
    if (tid < N1) {
        const int* o = s_off + tid * (C + 1);
        W = o[C] - o[0] + C;
        const int S = s_st[tid * C];
        U = s_st[tid * C + C - 1] + (o[C] - o[C - 1]) - S;
        if (U < 0) U += N;
        rS[tid] = S;
    }
    // inclusive block scans of W and U (blockDim.x = 1024 = 32 warps)
    const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    int wi = W, ui = U;
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, wi, o), c = __shfl_up_sync(0xffffffffu, ui, o);
        if (lane >= o) { wi += a; ui += c; }
    }
    if (lane == 31) { red[warp] = wi; red[32 + warp] = ui; }
    __syncthreads();
    int wbase = 0, ubase = 0;
    for (int w = 0; w < warp; ++w) { wbase += red[w]; ubase += red[32 + w]; }
    if (tid < N1) {
        wrun[tid + 1] = wbase + wi;
        urun[tid + 1] = ubase + ui;
    }
    if (tid == 0) {
        wrun[0] = urun[0] = 0;
        hdr[b] = make_int4(wstart[b], wlen[b], ustart[b], ulen[b]);
    }
    __syncthreads();
    float* awb = aw + wstart[b];
    int32_t* alb = alist + ustart[b];
    int32_t* asb = alist_sorted + ustart[b];
    for (int r = warp; r < N1; r += nw) {
        const int* o = s_off + r * (C + 1);
        const int o0 = o[0], nrun = o[C] - o0;
        // the run's weights (its columns are contiguous in w32), column c shifted by c slots:
        // each column is followed by one unused slot, so that the columns of a warp start on
        // spread-out shared-memory banks
        for (int i = lane; i < nrun; i += 32) {
            int c = 0;
            while (c + 1 < C && o[c + 1] - o0 <= i) ++c;
            awb[wrun[r] + i + c] = w32[o0 + i];
        }
        if (lane < C) awb[wrun[r] + (o[lane + 1] - o0) + lane] = 0.f;
        const int S = rS[r], Ur = urun[r + 1] - urun[r];
        for (int i = lane; i < Ur; i += 32) {
            int q = S + i;
            if (q >= N) q -= N;
            alb[urun[r] + i] = perm[q];
            asb[urun[r] + i] = q;
        }
    }
    for (int j = tid; j < NCOL; j += blockDim.x) {
        const int r = j / C, c = j - r * C;
        const int* o = s_off + r * (C + 1);
        const int woff = wrun[r] + (o[c] - o[0]) + c, n = o[c + 1] - o[c];
        int r0 = s_st[j] - rS[r];
        if (r0 < 0) r0 += N;
        const unsigned uoff = (unsigned)(urun[r] + (n ? r0 : 0));
        const int p = (r << log2) + C * b + c;
        cdesc[(size_t)b * NCOL + j] = make_uint2((unsigned)woff | ((unsigned)n << 16),
                                                 uoff | ((unsigned)(wide[p] != 0) << 31));
    }
    // zero the padding at the blocks' ends
    if (tid < 4) {
        const int w = wrun[N1] + tid, u = urun[N1] + tid;
        if (w < wlen[b]) awb[w] = 0.f;
        if (u < ulen[b]) {
            alb[u] = 0;
            asb[u] = 0;
        }
    }
}

// f_sorted[i] = f[perm[i]] (SORT) or out[perm[i]] = f[i]
template <bool SORT>
__global__ void k_permute_values(const float2* __restrict__ f, const int32_t* __restrict__ perm, int N,
                                 float2* __restrict__ out) {
    griddep_wait();
    griddep_launch();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        if (SORT) out[i] = f[perm[i]];
        else out[perm[i]] = f[i];
    }
}

using A1Fn = void (*)(A1Args);

struct A1Shape {
    int log1, C;
    A1Fn fn, fn_sorted;
    int smem;
};

template <int LOG1, int C> A1Shape shape_of() {
    return A1Shape{LOG1, C, k_apply_spread_fftA<LOG1, C, false>, k_apply_spread_fftA<LOG1, C, true>,
                   A1Layout<LOG1, C>::BYTES};
}

// the tile shapes: (log2 N1, C) with N1 C = 512 or 256 grid points per tile
const A1Shape* shapes(int* count) {
    static const A1Shape s[] = {shape_of<7, 4>(), shape_of<6, 8>(), shape_of<8, 2>(),
                                shape_of<6, 4>(), shape_of<7, 2>()};
    *count = (int)(sizeof(s) / sizeof(s[0]));
    return s;
}

bool shape_valid(const A1Shape& sh, int logMs) {
    const int log2 = logMs - sh.log1;
    return log2 >= 6 && log2 <= 12 && (1 << log2) >= sh.C;
}

}  // namespace

void apply2_config_shape(int id, int* log1, int* C) {
    int n;
    const A1Shape* s = shapes(&n);
    if (log1) *log1 = s[id].log1;
    if (C) *C = s[id].C;
}

int apply2_config_count() {
    int n;
    shapes(&n);
    return n;
}

bool apply2_config_valid(const Plan* p, int id) {
    int n;
    const A1Shape* s = shapes(&n);
    return id >= 0 && id < n && shape_valid(s[id], p->logMs);
}

int apply2_default_config(const Plan* p) {
    int n;
    const A1Shape* s = shapes(&n);
    // the expected weights of a tile, 2m N / M_sigma per grid point, within two thirds of the
    // staging buffer: 512 grid points per tile when they fit, else 256
    const double per_col = 2.0 * p->m * (double)p->N / (double)p->Ms;
    const int first = per_col * 512 <= A1_WMAX * 2.0 / 3.0 ? 0 : 3;
    for (int i = first; i < n; ++i)
        if (shape_valid(s[i], p->logMs)) return i;
    for (int i = 0; i < n; ++i)
        if (shape_valid(s[i], p->logMs)) return i;
    return -1;
}

int64_t apply2_max_tiles(const Plan* p) { return p->Ms / 256; }

int64_t apply2_weight_capacity(const Plan* p) {
    // every weight once, one skew slot per grid point, 3 padding slots per tile
    return p->nnz_cap + p->Ms + 4 * apply2_max_tiles(p);
}

int64_t apply2_list_capacity(const Plan* p) {
    // a node lies in the windows of at most (C + 2m)/C + 1 <= m + 2 runs (C >= 2), plus 3
    // padding entries per tile
    return p->N * ((int64_t)p->m + 2) + 4 * apply2_max_tiles(p);
}

// Lays out the tiles of the current shape (after precompute or a change of shape).
cudaError_t run_apply_layout(Plan* p, cudaStream_t s) {
    int n;
    const A1Shape* all = shapes(&n);
    const int id = p->apply_cfg >= 0 ? p->apply_cfg : apply2_default_config(p);
    if (id < 0 || !shape_valid(all[id], p->logMs)) return cudaErrorInvalidValue;
    const int log1 = all[id].log1, C = all[id].C, log2 = p->logMs - log1;
    const int tiles = (1 << log2) / C;
    if (tiles > apply2_max_tiles(p)) return cudaErrorInvalidValue;
    int32_t* wlen = p->lay_tmp;
    int32_t* ulen = wlen + tiles;
    int32_t* direct = ulen + tiles;
    int32_t* wstart = direct + tiles;
    int32_t* ustart = wstart + tiles;
    launch_begin(p, "layout_count", s);
    k_layout_count<<<tiles, 128, 0, s>>>(p->col_off, p->col_start, (int)p->N, log1, log2, C, wlen, ulen, direct);
    launch_end(p, s);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = run_exclusive_scan(p, wlen, wstart, tiles, s);
    if (e == cudaSuccess) e = run_exclusive_scan(p, ulen, ustart, tiles, s);
    if (e != cudaSuccess) return e;
    launch_begin(p, "layout_fill", s);
    k_layout_fill<<<tiles, 1024, 0, s>>>(p->col_off, p->col_start, p->w32, p->wide, p->perm, (int)p->N, log1, log2, C,
                                         wstart, ustart, wlen, ulen, direct, apply2_weight_capacity(p),
                                         apply2_list_capacity(p), p->lay_hdr, p->lay_cdesc, p->lay_w, p->lay_list,
                                         p->lay_list_sorted);
    launch_end(p, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    p->lay_cfg = id;
    return cudaSuccess;
}

cudaError_t run_sort_values(Plan* p, const float2* f, float2* out, cudaStream_t s) {
    const int N = (int)p->N;
    launch_begin(p, "sort_values", s);
    cudaError_t e = launch_pdl(k_permute_values<true>, dim3((N + 255) / 256), dim3(256), 0, s, f,
                               (const int32_t*)p->perm, N, out);
    launch_end(p, s);
    return e;
}

cudaError_t run_unsort_values(Plan* p, const float2* f, float2* out, cudaStream_t s) {
    const int N = (int)p->N;
    launch_begin(p, "unsort_values", s);
    cudaError_t e = launch_pdl(k_permute_values<false>, dim3((N + 255) / 256), dim3(256), 0, s, f,
                               (const int32_t*)p->perm, N, out);
    launch_end(p, s);
    return e;
}

cudaError_t run_apply2(Plan* p, const float2* f, bool sorted, float2* fhat, cudaStream_t s, int K, float2* Y) {
    int n;
    const A1Shape* all = shapes(&n);
    const int id = p->apply_cfg >= 0 ? p->apply_cfg : apply2_default_config(p);
    if (id < 0 || !shape_valid(all[id], p->logMs)) return cudaErrorInvalidValue;
    cudaError_t e;
    if (p->lay_cfg != id) {
        // a new B_opt or a new tile shape: lay the tiles out (plan data written in the stream,
        // so the next launch may not read it early)
        if ((e = run_apply_layout(p, s)) != cudaSuccess) return e;
        p->apply_clean = 0;
    }
    const A1Shape& sh = all[id];
    const int log1 = sh.log1, log2 = p->logMs - log1;
    A1Fn fn = sorted ? sh.fn_sorted : sh.fn;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem)) != cudaSuccess) return e;
    A1Args a;
    a.f = f; a.hdr = p->lay_hdr; a.cdesc = p->lay_cdesc; a.aw = p->lay_w;
    a.alist = sorted ? p->lay_list_sorted : p->lay_list;
    a.w32 = p->w32; a.wlo = p->wlo; a.wide = p->wide; a.perm = p->perm;
    a.col_start = p->col_start; a.col_off = p->col_off; a.Y = Y ? Y : (float2*)p->work;
    a.N = (int)p->N; a.log2 = log2;
    const int blocks = (1 << log2) / sh.C, threads = 256;
    launch_begin(p, "spread_fftA", s);
    if (p->apply_clean) {
        e = launch_pdl(fn, dim3(blocks, K), dim3(threads), (size_t)sh.smem, s, a);
    } else {
        // the first apply after set_nodes / precompute / a new layout: an ordinary launch, so
        // the early reads of plan data cannot overlap the kernels that wrote it
        fn<<<dim3(blocks, K), threads, sh.smem, s>>>(a);
        e = cudaGetLastError();
    }
    launch_end(p, s);
    if (e != cudaSuccess) return e;
    p->apply_clean = 1;
    return fft_passB_r8(a.Y, fhat, log1, log2, (int)p->M, p->kernel == INFFT_KERNEL_SYM, s, p, K);
}
