// Batched inverse NFFT: many independent problems of uneven size (M_p, N_p) in
// one plan, the paper's overdetermined direct inversion (Sec. 3.2.2) for each.
//
// Pattern and precompute: every problem is a plan of its own whose buffers are
// carved from one allocation, and each step is one launch over all problems: the
// pattern one CTA per problem (pattern.cu, k_batch_pattern), each solver tier one
// launch over the work items of all problems, numbered by a device prefix of the
// problems' counts (lsq.cu, run_precompute_batch), and the columns of more than 64
// nodes of all problems the blocked solver, four launches by column size.  Everything is
// stream-ordered on the caller's stream, so the whole precompute can be captured in
// a CUDA graph.
//
// Apply: two launches for the whole batch.  (1) Spreading, one CTA per tile of at
// most `cols` grid points of one problem, staged in shared memory; tiles are cut after
// the precompute so that each holds fewer than wblk + |I(l)|max weights (clustered
// nodes make some columns hundreds of nodes long).  (cols, wblk) is the batch's tile
// shape, chosen by measurement (infft_batch_tune_apply); every shape sums each column
// in the same order, so the shape changes the time and never the result.
// (2) One persistent CTA per SM takes problems by size: D^* F^* on the problem's
// grid of M_sigma = 2M points.  M is any even number, so the pruned DFT
//   h_k = sum_{l=-M}^{M-1} g_l w^{kl},  w = e^{-2 pi i/(2M)},  k = -M/2 .. M/2-1,
// is split into even and odd grid points, h_k = E_k + w^k O_k with length-M DFTs
//   E_k = sum_{n=-M/2}^{M/2-1} g_{2n} W^{kn},  O_k = sum_n g_{2n+1} W^{kn},  W = w^2,
// and each is evaluated as a chirp convolution (Bluestein, "A linear filtering
// approach to the computation of the discrete Fourier transform", 1970):
//   kn = (k^2 + n^2 - (k-n)^2)/2  =>  E_k = W^{k^2/2} sum_n (g_{2n} W^{n^2/2}) W^{-(k-n)^2/2},
// a cyclic convolution of length L = 2^ceil(log2(2M-1)) done with in-place
// radix-8 transforms in shared memory: a decimation-in-frequency forward
// transform (natural order in, digit-reversed out), a pointwise product with
// the transform of the chirp (precomputed per problem in the same digit-reversed
// order) and a decimation-in-time inverse (digit-reversed in, natural out).
// W^{n^2/2} = e^{-i pi (n^2 mod 2M)/M} is evaluated on the exactly reduced integer.
// When 3M - 1 <= 16384 the even/odd split is not needed: with kl = (k^2 + l^2 -
// (k-l)^2)/2 directly, h_k = w^{k^2/2} sum_l (g_l w^{l^2/2}) w^{-(k-l)^2/2} is one
// cyclic convolution of length L >= 3M - 1 (the 2M inputs and M outputs do not
// alias), two transforms instead of four.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "fft_device.cuh"
#include "plan.h"
#include "spread_device.cuh"

namespace {

constexpr int BATCH_FFT_THREADS = 1024;
constexpr int TW_LOG = 14;
constexpr int TW_N = 1 << TW_LOG;                 // twiddle table e^{-2 pi i t / TW_N}
constexpr int BATCH_MMAX = TW_N / 2;              // 2M - 1 <= TW_N
constexpr int BATCH_STASH = BATCH_MMAX / BATCH_FFT_THREADS;

struct BatchProblem {
    const float* w32;
    const double* w64;
    float* wlo;            // low parts fp32(w64 - w32) of the float-float spreading
    const uint8_t* wide;
    const int32_t* perm;
    const int32_t* col_start;
    const int32_t* col_count;
    const int32_t* col_off;
    const float2* bhat;    // L values: the chirp's transform, digit-reversed
    int64_t f_off, fhat_off, g_off;
    int N, M, logL, sym;
    int full;              // 1: one convolution over all 2M grid points (3M - 1 <= TW_N)
};

INFFT_HD int pad16(int i) { return i + (i >> 4); }   // one padding slot per 16 entries

// W^{n^2/2} = e^{-i pi (n^2 mod 2M)/M} for n = idx - M/2
INFFT_D float2 chirp(int idx, int M) {
    const int n = idx - M / 2;
    const int q = (n * n) % (2 * M);
    float s, c;
    sincospif(-(float)q / (float)M, &s, &c);
    return make_float2(c, s);
}

// w^{t^2/2} = e^{-i pi (t^2 mod 4M)/(2M)} for an integer t, w = e^{-2 pi i/(2M)}
INFFT_D float2 chirp4(int t, int M) {
    const int q = (t * t) % (4 * M);
    float s, c;
    sincospif(-(float)q / (float)(2 * M), &s, &c);
    return make_float2(c, s);
}

// Twiddles of the in-CTA transforms: e^{-2 pi i t/TW_N} = C[t >> 7] F[t & 127]
// from two 128-entry tables in shared memory (filled once per CTA from the global
// table), and the powers w^r, r < 8, of a butterfly's w by products of depth <= 3.
struct TwTables {
    float2 c[128], f[128];
};

INFFT_D void tw_tables_load(TwTables* t, const float2* __restrict__ tw) {
    for (int j = threadIdx.x; j < 128; j += blockDim.x) {
        t->c[j] = tw[j << 7];
        t->f[j] = tw[j];
    }
}

INFFT_D float2 tw_of(const TwTables* t, int e) { return cmul(t->c[e >> 7], t->f[e & 127]); }

template <int R> INFFT_D void tw_powers(float2 w1, float2* w) {   // w[r] = w1^r, r = 1 .. R-1
    w[1] = w1;
    if (R > 2) {
        w[2] = cmul(w1, w1);
        w[3] = cmul(w[2], w1);
    }
    if (R > 4) {
        w[4] = cmul(w[2], w[2]);
        w[5] = cmul(w[4], w1);
        w[6] = cmul(w[4], w[2]);
        w[7] = cmul(w[4], w[3]);
    }
}

// One in-place decimation-in-frequency radix-R stage on blocks of S entries:
// butterfly (block, o) reads x_r = a[base + o + r S/R], transforms, multiplies
// X_r by e^{-2 pi i o r / S} and writes back to the same entries.
template <int R>
INFFT_D void dif_stage(float2* buf, int L, int S, const TwTables* tw) {
    const int h = S / R, lh = __ffs(h) - 1, nbf = L / R, ts = TW_N / S;
    for (int bf = threadIdx.x; bf < nbf; bf += blockDim.x) {
        const int base = ((bf >> lh) * S) + (bf & (h - 1));
        const int o = bf & (h - 1);
        float2 x[R], w[R];
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = buf[pad16(base + r * h)];
        dft_r<-1>(x, int_constant_tag<R>());
        tw_powers<R>(tw_of(tw, o * ts), w);
#pragma unroll
        for (int r = 1; r < R; ++r) x[r] = cmul(x[r], w[r]);
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pad16(base + r * h)] = x[r];
    }
}

// The transpose of dif_stage with conjugate twiddles (decimation in time, +i).
template <int R>
INFFT_D void dit_stage_inv(float2* buf, int L, int S, const TwTables* tw) {
    const int h = S / R, lh = __ffs(h) - 1, nbf = L / R, ts = TW_N / S;
    for (int bf = threadIdx.x; bf < nbf; bf += blockDim.x) {
        const int base = ((bf >> lh) * S) + (bf & (h - 1));
        const int o = bf & (h - 1);
        float2 x[R], w[R];
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = buf[pad16(base + r * h)];
        tw_powers<R>(tw_of(tw, o * ts), w);
#pragma unroll
        for (int r = 1; r < R; ++r) x[r] = cmul(x[r], make_float2(w[r].x, -w[r].y));
        dft_r<1>(x, int_constant_tag<R>());
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pad16(base + r * h)] = x[r];
    }
}

// Forward transform of L = 2^logL entries (natural order in, digit-reversed out).
INFFT_D void cta_dif_forward(float2* buf, int logL, const TwTables* tw) {
    const int L = 1 << logL;
    int S = L;
    for (int i = 0; i < logL / 3; ++i) {
        dif_stage<8>(buf, L, S, tw);
        __syncthreads();
        S >>= 3;
    }
    if (logL % 3 == 1) { dif_stage<2>(buf, L, S, tw); __syncthreads(); }
    if (logL % 3 == 2) { dif_stage<4>(buf, L, S, tw); __syncthreads(); }
}

// Inverse transform without the 1/L (digit-reversed in, natural order out).
INFFT_D void cta_dit_inverse(float2* buf, int logL, const TwTables* tw) {
    const int L = 1 << logL;
    int S = 1;
    if (logL % 3 == 1) { S = 2; dit_stage_inv<2>(buf, L, S, tw); __syncthreads(); }
    if (logL % 3 == 2) { S = 4; dit_stage_inv<4>(buf, L, S, tw); __syncthreads(); }
    for (int i = 0; i < logL / 3; ++i) {
        S <<= 3;
        dit_stage_inv<8>(buf, L, S, tw);
        __syncthreads();
    }
}

// buf <- L * (a (*) b) for a in buf (natural order) and bhat = DIF(b).
INFFT_D void chirp_convolve(float2* buf, int logL, const float2* __restrict__ bhat, const TwTables* tw) {
    const int L = 1 << logL;
    cta_dif_forward(buf, logL, tw);
    for (int i = threadIdx.x; i < L; i += blockDim.x) buf[pad16(i)] = cmul(buf[pad16(i)], __ldg(bhat + i));
    __syncthreads();
    cta_dit_inverse(buf, logL, tw);
}

// Per problem: bhat = DIF(b), b_d = W^{-d^2/2} = e^{+i pi (d^2 mod 2M)/M} for |d| < M
// placed cyclically (d mod L), zero elsewhere.
__global__ void __launch_bounds__(BATCH_FFT_THREADS)
k_batch_chirp(const BatchProblem* __restrict__ probs, float2* __restrict__ bhat_all,
              const int64_t* __restrict__ bhat_off, const float2* __restrict__ tw) {
    extern __shared__ __align__(16) float2 sm[];
    __shared__ TwTables twt;
    tw_tables_load(&twt, tw);
    const BatchProblem pr = probs[blockIdx.x];
    const int M = pr.M, L = 1 << pr.logL;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        if (pr.full) {
            // beta_s = w^{-(s + M/2)^2/2} for s = k' - j in (-2M, M), placed cyclically
            if (i < M || i > L - 2 * M) {
                const int t = (i < M ? i : i - L) + M / 2;
                const int q = (t * t) % (4 * M);
                float sn, cs;
                sincospif((float)q / (float)(2 * M), &sn, &cs);
                v = make_float2(cs, sn);
            }
        } else if (i < M || i > L - M) {   // |d| < M
            const int d = i < M ? i : i - L;
            const int q = (d * d) % (2 * M);
            float sn, cs;
            sincospif((float)q / (float)M, &sn, &cs);
            v = make_float2(cs, sn);
        }
        sm[pad16(i)] = v;
    }
    __syncthreads();
    cta_dif_forward(sm, pr.logL, &twt);
    float2* out = bhat_all + bhat_off[blockIdx.x];
    for (int i = threadIdx.x; i < L; i += blockDim.x) out[i] = sm[pad16(i)];
}

// Tiles of the batched spreading, the autotuned part of the batched apply.  A tile
// shape is (cols, wblk), both powers of two: grid point p of a problem starts a tile
// when p is a multiple of cols or when its weight offset enters a new block of wblk
// entries, so a tile has at most cols grid points (one thread each) and fewer than
// wblk + |I(l)|max weights.  The shapes are the tuner's candidates (the default is
// the fixed rule, 128 grid points and 2048 weights).  Every shape gives the same
// sums: each column is summed in one order that depends on the grid point only.
struct TileShape {
    int log_cols, log_wblk;
};
constexpr TileShape TILE_SHAPES[] = {{6, 10}, {6, 11}, {6, 12}, {7, 10}, {7, 11}, {7, 12},
                                     {8, 11}, {8, 12}, {8, 13}, {9, 12}, {9, 13}};
constexpr int TILE_SHAPE_COUNT = (int)(sizeof(TILE_SHAPES) / sizeof(TILE_SHAPES[0]));
constexpr int TILE_SHAPE_DEFAULT = 4;
constexpr int TILE_SCAN_THREADS = 1024;

INFFT_D bool tile_start(const int32_t* __restrict__ col_off, int p, int lc, int lw) {
    return (p & ((1 << lc) - 1)) == 0 || (col_off[p] >> lw) != (col_off[p - 1] >> lw);
}

// Per problem (one CTA): its number of tiles.
__global__ void __launch_bounds__(TILE_SCAN_THREADS)
k_tile_count(const BatchProblem* __restrict__ probs, int lc, int lw, int32_t* __restrict__ count) {
    const BatchProblem pr = probs[blockIdx.x];
    const int Ms = 2 * pr.M;
    int c = 0;
    for (int p = threadIdx.x; p < Ms; p += blockDim.x) c += tile_start(pr.col_off, p, lc, lw);
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ int red[TILE_SCAN_THREADS / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < TILE_SCAN_THREADS / 32; ++w) t += red[w];
        count[blockIdx.x] = t;
    }
}

// Exclusive prefix of the P tile counts (one CTA); off[P] = total.
__global__ void __launch_bounds__(1024) k_tile_prefix(const int32_t* __restrict__ count, int P, int32_t* __restrict__ off) {
    __shared__ int32_t part[1024];
    const int per = (P + 1023) / 1024;
    const int a = threadIdx.x * per, b = min(a + per, P);
    int32_t sum = 0;
    for (int i = a; i < b; ++i) sum += count[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const int32_t v = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int i = a; i < b; ++i) {
        off[i] = run;
        run += count[i];
    }
    if (threadIdx.x == 1023) off[P] = part[1023];
}

// Per problem (one CTA): writes its tiles at its offset, two int4 each: (problem,
// first grid point, end grid point, first node S) and (first weight, end weight,
// node window U, 0); thread t scans a contiguous run of grid points.
__global__ void __launch_bounds__(TILE_SCAN_THREADS)
k_tile_fill(const BatchProblem* __restrict__ probs, int lc, int lw, const int32_t* __restrict__ off,
            int4* __restrict__ tiles) {
    const BatchProblem pr = probs[blockIdx.x];
    const int Ms = 2 * pr.M;
    const int per = (Ms + TILE_SCAN_THREADS - 1) / TILE_SCAN_THREADS;
    const int a = min((int)threadIdx.x * per, Ms), b = min(a + per, Ms);
    int c = 0;
    for (int p = a; p < b; ++p) c += tile_start(pr.col_off, p, lc, lw);
    __shared__ int part[TILE_SCAN_THREADS];
    part[threadIdx.x] = c;
    __syncthreads();
    for (int d = 1; d < TILE_SCAN_THREADS; d <<= 1) {
        const int v = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int pos = off[blockIdx.x] + part[threadIdx.x] - c;
    for (int p = a; p < b; ++p) {
        if (!tile_start(pr.col_off, p, lc, lw)) continue;
        int q = p + 1;   // the tile ends at the next start
        while (q < Ms && !tile_start(pr.col_off, q, lc, lw)) ++q;
        // the tile's weights [w0, w1) and its window of U sorted nodes from S (mod N)
        const int S = pr.col_start[p];
        int U = pr.col_start[q - 1] + pr.col_count[q - 1] - S;
        if (U < 0) U += pr.N;
        tiles[2 * pos] = make_int4((int)blockIdx.x, p, q, S);
        tiles[2 * pos + 1] = make_int4(pr.col_off[p], pr.col_off[q], U, 0);
        ++pos;
    }
}

// g_l of grid point p in its one summation order, whatever the tile: the entries
// i = k0, k0 + 1, .., n - 1, 0, .., k0 - 1 with k0 = (p mod 32) mod n, one fmaf per entry
// and component (float-float, w32 + wlo, for wide columns).  Starting each column at
// its grid point's lane spreads a warp's shared-memory accesses over the banks
// (neighbouring columns sit |I(l)| weights apart).  From staged data: wc and fc are
// the column's weights and node values in shared memory.
INFFT_D float2 col_sum_staged(const float* wc, const float2* fc, int n, int k0) {
    float re = 0, im = 0;
    for (int k = k0; k < n; ++k) {   // the same order as one walk from k0 with wrap-around
        const float wi = wc[k];
        const float2 v = fc[k];
        re = fmaf(wi, v.x, re);
        im = fmaf(wi, v.y, im);
    }
    for (int k = 0; k < k0; ++k) {
        const float wi = wc[k];
        const float2 v = fc[k];
        re = fmaf(wi, v.x, re);
        im = fmaf(wi, v.y, im);
    }
    return make_float2(re, im);
}

// The same sum by direct loads (node s + k of the sorted order is f[perm[(s + k) mod N]]).
INFFT_D float2 col_sum_direct(const float2* __restrict__ f, const float* __restrict__ w32,
                              const float* __restrict__ wlo, bool wide_col, const int32_t* __restrict__ perm,
                              int n, int s, int off, int N, int k0) {
    int k = k0, q = s + k0;
    if (q >= N) q -= N;
    if (wide_col) {
        FFSum acc;
        for (int i = 0; i < n; ++i) {
            acc.add(w32[off + k], wlo[off + k], f[perm[q]]);
            if (++k == n) k = 0, q = s - 1;
            if (++q >= N) q -= N;
        }
        return acc.value();
    }
    float re = 0, im = 0;
    for (int i = 0; i < n; ++i) {
        const float wi = w32[off + k];
        const float2 v = f[perm[q]];
        re = fmaf(wi, v.x, re);
        im = fmaf(wi, v.y, im);
        if (++k == n) k = 0, q = s - 1;
        if (++q >= N) q -= N;
    }
    return make_float2(re, im);
}

// Spreading of all problems with tiles of shape (2^LC grid points, 2^LW weight
// blocks): CTA t spreads tile t (problem, [p0, p1)) into the problem's slice of
// g_all; CTAs beyond the number of tiles return.  The tile record carries the
// tile's weight range and node window, so the weights and node indices are
// requested together with the threads' column data (two dependent load phases per
// tile: weights and indices, then node values).  A node window longer than the
// staging buffer (the densest clusters) is staged in pieces, twice: the first sweep
// adds each column's entries k0 .. n-1, the second its entries 0 .. k0-1, which keeps
// the one summation order.  Wide columns, columns outside the window and tiles whose
// weights do not fit (a column above HUGE_NMAX nodes) are summed by direct loads, in
// the same order.  (A persistent, two-stage software-pipelined variant was slower:
// 1.48 ms against 1.10 ms on the batched workload, at half the resident threads per SM.)
template <int LC, int LW>
__global__ void __launch_bounds__(1 << LC)
k_batch_spread(const BatchProblem* __restrict__ probs, const int4* __restrict__ tiles,
               const int32_t* __restrict__ ntiles, const float2* __restrict__ f, float2* __restrict__ g_all) {
    constexpr int COLS = 1 << LC;
    constexpr int WMAX = (1 << LW) + HUGE_NMAX + 8;       // wblk + the largest solved column + alignment
    constexpr int UMAX = COLS * 8 > 1024 ? COLS * 8 : 1024;
    constexpr int UPT = UMAX / COLS;
    extern __shared__ __align__(16) unsigned char bsp_smem[];
    float* ws = (float*)bsp_smem;                       // WMAX weights (a multiple of 16 bytes)
    float2* fu = (float2*)(bsp_smem + WMAX * 4);        // UMAX node values
    if ((int)blockIdx.x >= *ntiles) return;
    const int4 ra = tiles[2 * blockIdx.x], rb = tiles[2 * blockIdx.x + 1];
    const int p0 = ra.y, p1 = ra.z, S = ra.w, w0 = rb.x, w1 = rb.y, U = rb.z;
    const BatchProblem& pr = probs[ra.x];
    const int N = pr.N;
    const float2* fp = f + pr.f_off;
    float2* g = g_all + pr.g_off;
    const float* w32 = pr.w32;
    const int32_t* perm = pr.perm;
    const int wb = w0 & ~3, we = (w1 + 3) & ~3;
    const bool staged = (we - wb) <= WMAX && U <= N;       // block-uniform
    const bool one_piece = U <= UMAX;
    int pq[UPT];
    // the staging rounds this warp takes part in (warp-uniform: its lanes' first q is the warp's base)
    const int wbase = threadIdx.x & ~31;
    const int nu = U > wbase ? min(UPT, (U - wbase + COLS - 1) / COLS) : 0;
    if (staged) {
        for (int v = threadIdx.x; v < (we - wb) / 4; v += COLS) cp_async16(ws + 4 * v, w32 + wb + 4 * v);
        if (one_piece) {
#pragma unroll
            for (int u = 0; u < UPT; ++u) {
                if (u < nu) {
                    const int q = threadIdx.x + u * COLS;
                    int gq = S + q;
                    if (gq >= N) gq -= N;
                    pq[u] = q < U ? perm[gq] : 0;
                }
            }
        }
    }
    const int p = p0 + threadIdx.x;
    const bool live = p < p1;
    const int n = live ? pr.col_count[p] : 0;
    const int s = live ? pr.col_start[p] : 0;
    const int off = live ? pr.col_off[p] : 0;
    const bool wide_col = live && pr.wide[p];
    int k0 = p & 31;                  // (p mod 32) mod n, by subtraction (n is mostly above 31)
    if (n == 0) k0 = 0;
    else while (k0 >= n) k0 -= n;
    int r0 = s - S;
    if (r0 < 0) r0 += N;
    const bool direct = !staged || wide_col || (n > 0 && r0 + n > U);
    float2 acc = make_float2(0.f, 0.f);
    if (staged && one_piece) {
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
            const int q = threadIdx.x + u * COLS;
            if (u < nu && q < U) cp_async8(fu + q, fp + pq[u]);
        }
        cp_async_wait_all();
        __syncthreads();
        if (live && !direct) acc = col_sum_staged(ws + (off - wb), fu + r0, n, k0);
    } else if (staged) {
        const float* wc = ws + (off - wb);
        float re = 0, im = 0;
        for (int sweep = 0; sweep < 2; ++sweep) {
            // window positions of the sweep's entries: [r0 + k0, r0 + n), then [r0, r0 + k0)
            const int lo = sweep == 0 ? r0 + k0 : r0, hi = sweep == 0 ? r0 + n : r0 + k0;
            for (int c0 = 0; c0 < U; c0 += UMAX) {
                __syncthreads();   // the previous piece is consumed
                const int len = min(UMAX, U - c0);
                for (int q = threadIdx.x; q < len; q += COLS) {
                    int gq = S + c0 + q;
                    if (gq >= N) gq -= N;
                    cp_async8(fu + q, fp + perm[gq]);
                }
                cp_async_wait_all();
                __syncthreads();
                if (live && !direct) {
                    const int a = max(lo, c0), e = min(hi, c0 + len);
                    for (int r = a; r < e; ++r) {
                        const float wi = wc[r - r0];
                        const float2 v = fu[r - c0];
                        re = fmaf(wi, v.x, re);
                        im = fmaf(wi, v.y, im);
                    }
                }
            }
        }
        acc = make_float2(re, im);
    }
    if (!live) return;
    g[p] = direct ? col_sum_direct(fp, w32, pr.wlo, wide_col, perm, n, s, off, N, k0) : acc;
}

// shared memory of shape (LC, LW): the staged weights and node values
template <int LC, int LW> constexpr size_t batch_spread_smem() {
    return (size_t)((1 << LW) + HUGE_NMAX + 8) * 4 + (size_t)((1 << LC) * 8 > 1024 ? (1 << LC) * 8 : 1024) * 8;
}

template <int LC, int LW>
cudaError_t launch_spread_shape(unsigned grid, const BatchProblem* probs, const int4* tiles, const int32_t* ntiles,
                                const float2* f, float2* g, cudaStream_t s) {
    constexpr size_t sm = batch_spread_smem<LC, LW>();
    static_assert(((1 << LW) + HUGE_NMAX + 8) * 4 % 16 == 0, "node values 16-byte aligned");
    cudaError_t e = cudaFuncSetAttribute(k_batch_spread<LC, LW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_batch_spread<LC, LW><<<grid, 1 << LC, sm, s>>>(probs, tiles, ntiles, f, g);
    return cudaGetLastError();
}

cudaError_t launch_batch_spread(int shape, unsigned grid, const BatchProblem* probs, const int4* tiles,
                                const int32_t* ntiles, const float2* f, float2* g, cudaStream_t s) {
    switch (shape) {
#define INFFT_SPREAD_SHAPE(ID, LC, LW)                                                   \
    case ID:                                                                             \
        static_assert(TILE_SHAPES[ID].log_cols == LC && TILE_SHAPES[ID].log_wblk == LW, ""); \
        return launch_spread_shape<LC, LW>(grid, probs, tiles, ntiles, f, g, s);
        INFFT_SPREAD_SHAPE(0, 6, 10)
        INFFT_SPREAD_SHAPE(1, 6, 11)
        INFFT_SPREAD_SHAPE(2, 6, 12)
        INFFT_SPREAD_SHAPE(3, 7, 10)
        INFFT_SPREAD_SHAPE(4, 7, 11)
        INFFT_SPREAD_SHAPE(5, 7, 12)
        INFFT_SPREAD_SHAPE(6, 8, 11)
        INFFT_SPREAD_SHAPE(7, 8, 12)
        INFFT_SPREAD_SHAPE(8, 8, 13)
        INFFT_SPREAD_SHAPE(9, 9, 12)
        INFFT_SPREAD_SHAPE(10, 9, 13)
#undef INFFT_SPREAD_SHAPE
        default:
            return cudaErrorInvalidValue;
    }
}

// D^* F^* of every problem's grid (pruned to its M central frequencies): one CTA
// per SM takes the problems in the order given (largest first) by a ticket.
__global__ void __launch_bounds__(BATCH_FFT_THREADS, 1)
k_batch_fft(const BatchProblem* __restrict__ probs, int P, const int32_t* __restrict__ order,
            const float2* __restrict__ g_all, float2* __restrict__ fhat, const float2* __restrict__ tw,
            int32_t* __restrict__ ticket) {
    extern __shared__ __align__(16) float2 sm[];
    float2* buf = sm;                    // pad16(L) <= pad16(TW_N)
    float2* gO = sm + pad16(TW_N);       // odd grid values, M <= BATCH_MMAX
    __shared__ int s_job;
    __shared__ TwTables twt;
    tw_tables_load(&twt, tw);
    for (;;) {
        if (threadIdx.x == 0) s_job = atomicAdd(ticket, 1);
        __syncthreads();
        const int job = s_job;
        __syncthreads();
        if (job >= P) break;
        const BatchProblem pr = probs[order[job]];
        const int M = pr.M, L = 1 << pr.logL;
        const float dk = 1.0f / (float)(2 * M);
        float2* out = fhat + pr.fhat_off;
        if (pr.full) {
            const float2* gp = g_all + pr.g_off;
            for (int j = threadIdx.x; j < 2 * M; j += blockDim.x) buf[pad16(j)] = cmul(gp[j], chirp4(j - M, M));
            for (int i = 2 * M + threadIdx.x; i < L; i += blockDim.x) buf[pad16(i)] = make_float2(0.f, 0.f);
            __syncthreads();
            chirp_convolve(buf, pr.logL, pr.bhat, &twt);
            const float invL = 1.0f / (float)L;
            for (int k = threadIdx.x; k < M; k += blockDim.x) {
                const float2 h = cscale(cmul(buf[pad16(k)], chirp4(k - M / 2, M)), invL);
                out[k] = cscale(h, (pr.sym && k == 0) ? 0.0f : dk);
            }
            __syncthreads();
            continue;
        }
        const float4* g4 = (const float4*)(g_all + pr.g_off);   // (g_{2n'}, g_{2n'+1})
        for (int n = threadIdx.x; n < M; n += blockDim.x) {
            const float4 v = g4[n];
            buf[pad16(n)] = cmul(make_float2(v.x, v.y), chirp(n, M));
            gO[n] = make_float2(v.z, v.w);
        }
        for (int i = M + threadIdx.x; i < L; i += blockDim.x) buf[pad16(i)] = make_float2(0.f, 0.f);
        __syncthreads();
        chirp_convolve(buf, pr.logL, pr.bhat, &twt);
        const float invL = 1.0f / (float)L;
        float2 X0[BATCH_STASH];
#pragma unroll
        for (int j = 0; j < BATCH_STASH; ++j) {
            const int k = threadIdx.x + j * BATCH_FFT_THREADS;
            X0[j] = k < M ? cscale(cmul(buf[pad16(k)], chirp(k, M)), invL) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int n = threadIdx.x; n < M; n += blockDim.x) buf[pad16(n)] = cmul(gO[n], chirp(n, M));
        for (int i = M + threadIdx.x; i < L; i += blockDim.x) buf[pad16(i)] = make_float2(0.f, 0.f);
        __syncthreads();
        chirp_convolve(buf, pr.logL, pr.bhat, &twt);
#pragma unroll
        for (int j = 0; j < BATCH_STASH; ++j) {
            const int k = threadIdx.x + j * BATCH_FFT_THREADS;
            if (k < M) {
                const float2 X1 = cscale(cmul(buf[pad16(k)], chirp(k, M)), invL);
                float s, c;
                sincospif(-(float)(k - M / 2) / (float)M, &s, &c);   // w^k
                const float2 h = cadd(X0[j], cmul(make_float2(c, s), X1));
                out[k] = cscale(h, (pr.sym && k == 0) ? 0.0f : dk);
            }
        }
        __syncthreads();
    }
}

// Per problem: nnz, the pattern and precompute counters and sum_l J_l.
__global__ void k_batch_info(const int32_t* const* __restrict__ counters, const int32_t* const* __restrict__ col_off,
                             const double* const* __restrict__ J, const int32_t* __restrict__ Ms,
                             double* __restrict__ out) {
    const int p = blockIdx.x;
    const int n = Ms[p];
    double sum = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) sum += J[p][i];
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        double* o = out + 8 * (size_t)p;
        o[0] = (double)col_off[p][n];
        o[1] = (double)counters[p][CNT_MAX_COLUMN];
        o[2] = (double)counters[p][CNT_EMPTY];
        o[3] = (double)counters[p][CNT_BAD_NODES];
        o[4] = (double)counters[p][CNT_FALLBACK];
        o[5] = (double)counters[p][CNT_UNSUPPORTED];
        o[6] = t;
        o[7] = (double)counters[p][CNT_HUGE_LIST];
    }
}

bool on_device(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int log2_ceil(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

}  // namespace

struct infft_batch_s {
    int device = 0;
    int64_t P = 0, sumN = 0, sumM = 0, sumG = 0, sumL = 0;
    int m = 0, kernel = INFFT_KERNEL_FULL, sms = 0, huge_slots = 0, huge_nmax = 0;
    double sigma = 2.0, tau = 1e-12;
    std::vector<int64_t> M, N, noff, moff;
    std::vector<Plan*> plans;
    void* arena = nullptr;          // all members' buffers
    double* x_all = nullptr;        // sum N nodes
    float2* g_all = nullptr;        // sum 2M grid values
    float2* bhat = nullptr;         // sum L chirp transforms
    float2* tw = nullptr;           // TW_N twiddles
    float2* stage_f = nullptr;      // host staging: sum N
    float2* stage_fhat = nullptr;   // host staging: sum M
    BatchProblem* probs = nullptr;  // P apply descriptors
    void* huge_probs = nullptr;     // P large-column descriptors
    int32_t* job_off = nullptr;     // P + 1
    int32_t* job_order = nullptr;   // sum M_sigma: blocked-solver jobs, largest first
    int32_t* job_work = nullptr;    // HUGE_NMAX + 8: size buckets, four tickets and three splits
    double* huge_scratch = nullptr;
    int32_t* order = nullptr;       // problems by decreasing size
    int32_t* ticket = nullptr;
    int4* tiles = nullptr;          // two int4 per spreading tile (see k_tile_fill)
    int32_t* tile_count = nullptr;  // P counts, then P + 1 offsets
    int32_t* tile_off = nullptr;
    int64_t max_tiles = 0;
    int tile_shape = TILE_SHAPE_DEFAULT;   // the spreading's tile shape (TILE_SHAPES)
    int64_t shape_tiles[TILE_SHAPE_COUNT] = {};   // the tile-count bound of each shape (the launch's grid)
    PatternArgs* pat_args = nullptr;   // P pattern descriptors (one launch for every problem's pattern)
    void* tier_args = nullptr;         // P solver-tier descriptors (one launch per tier)
    int32_t* pat_order = nullptr;      // problems by decreasing N (the pattern's CTAs take them in order)
    int32_t* tier_tile_off = nullptr;  // P + 1: prefix of the problems' 32-column tiles
    int32_t* tier_work = nullptr;      // 5 (P + 1): prefixes of the routed lists
    int64_t total_tiles32 = 0;
    const int32_t** d_counters = nullptr;
    const int32_t** d_col_off = nullptr;
    const double** d_J = nullptr;
    int32_t* d_Ms = nullptr;
    double* d_info = nullptr;       // 8 P
    int nodes_set = 0, precomputed = 0;
    cudaStream_t last_stream = nullptr;
};

namespace {

// The spreading tiles of the batch's tile shape, cut from the weight offsets.
cudaError_t build_tiles(infft_batch_t b, cudaStream_t s) {
    const TileShape sh = TILE_SHAPES[b->tile_shape];
    k_tile_count<<<(unsigned)b->P, TILE_SCAN_THREADS, 0, s>>>(b->probs, sh.log_cols, sh.log_wblk, b->tile_count);
    k_tile_prefix<<<1, 1024, 0, s>>>(b->tile_count, (int)b->P, b->tile_off);
    k_tile_fill<<<(unsigned)b->P, TILE_SCAN_THREADS, 0, s>>>(b->probs, sh.log_cols, sh.log_wblk, b->tile_off,
                                                             b->tiles);
    count_launches(3);
    return cudaGetLastError();
}

void batch_free(infft_batch_t b) {
    for (Plan* p : b->plans) delete p;
    void* bufs[] = {b->arena, b->x_all, b->g_all, b->bhat, b->tw, b->stage_f, b->stage_fhat, b->probs,
                    b->huge_probs, b->job_off, b->job_order, b->job_work, b->huge_scratch, b->order, b->ticket, b->tiles, b->tile_count, b->tile_off,
                    (void*)b->pat_args, b->tier_args, b->pat_order, b->tier_tile_off, b->tier_work,
                    (void*)b->d_counters, (void*)b->d_col_off, (void*)b->d_J, b->d_Ms, b->d_info};
    for (void* p : bufs)
        if (p) cudaFree(p);
    delete b;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

infft_status cuda_err(cudaError_t e, const char* what) {
    return set_error(e == cudaErrorMemoryAllocation ? INFFT_ENOMEM : INFFT_ECUDA, "%s: %s", what,
                     cudaGetErrorString(e));
}

}  // namespace

extern "C" {

infft_status infft_batch_create(int64_t P, const int64_t* M, const int64_t* N, double sigma, int m, int kernel,
                                double tau, infft_batch_t* out) {
    if (!out) return set_error(INFFT_EINVAL, "out is NULL");
    *out = nullptr;
    if (P < 1 || P > (1 << 24)) return set_error(INFFT_EINVAL, "P must be in [1, 2^24] (got %lld)", (long long)P);
    if (!M || !N) return set_error(INFFT_EINVAL, "M and N must not be NULL");
    if (sigma != 2.0) return set_error(INFFT_EUNSUPPORTED, "batched plans use sigma = 2 (got %g)", sigma);
    if (kernel != INFFT_KERNEL_FULL && kernel != INFFT_KERNEL_SYM)
        return set_error(INFFT_EINVAL, "kernel must be INFFT_KERNEL_FULL or INFFT_KERNEL_SYM (got %d)", kernel);
    if (!(tau >= 0.0 && tau < 1.0)) return set_error(INFFT_EINVAL, "tau must be in [0, 1) (got %g)", tau);
    for (int64_t i = 0; i < P; ++i) {
        if (M[i] < 4 || (M[i] & 1) || M[i] > BATCH_MMAX)
            return set_error(INFFT_EINVAL, "problem %lld: M must be even in [4, %d] (got %lld)", (long long)i,
                             BATCH_MMAX, (long long)M[i]);
        if (N[i] < 1 || (double)N[i] * (2.0 * m + 1.0) >= 2147483647.0)
            return set_error(INFFT_EINVAL, "problem %lld: N = %lld out of range", (long long)i, (long long)N[i]);
        if (m < 1 || 2 * (int64_t)m >= 2 * M[i])
            return set_error(INFFT_EINVAL, "problem %lld: need m >= 1 and 2m < M_sigma", (long long)i);
    }
    {
        // every index of the batch's concatenated arrays (nodes, grid points, weights of
        // one problem, spreading tiles) must fit the kernels' 32-bit arithmetic
        int64_t sn = 0, sg = 0;
        for (int64_t i = 0; i < P; ++i) {
            sn += N[i];
            sg += 2 * M[i];
        }
        if (sn >= (int64_t(1) << 31) || sg >= (int64_t(1) << 31))
            return set_error(INFFT_EUNSUPPORTED, "batch too large: sum N = %lld, sum M_sigma = %lld (each < 2^31)",
                             (long long)sn, (long long)sg);
    }
    int dev = 0, sms = 0;
    cudaError_t qe = cudaGetDevice(&dev);
    if (qe == cudaSuccess) qe = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (qe != cudaSuccess || sms <= 0)
        return set_error(INFFT_ECUDA, "cannot query the device's multiprocessor count: %s",
                         qe != cudaSuccess ? cudaGetErrorString(qe) : "count <= 0");
    infft_batch_t b = new infft_batch_s();
    b->device = dev;
    b->sms = sms;
    b->P = P; b->sigma = sigma; b->m = m; b->kernel = kernel; b->tau = tau;
    b->M.assign(M, M + P);
    b->N.assign(N, N + P);
    b->noff.resize(P + 1);
    b->moff.resize(P + 1);
    b->noff[0] = b->moff[0] = 0;
    std::vector<int64_t> goff(P + 1, 0), loff(P + 1, 0);
    std::vector<int> logL(P), full(P);
    int64_t maxN = 0;
    for (int64_t i = 0; i < P; ++i) {
        b->noff[i + 1] = b->noff[i] + N[i];
        b->moff[i + 1] = b->moff[i] + M[i];
        goff[i + 1] = goff[i] + 2 * M[i];
        full[i] = 3 * M[i] - 1 <= TW_N;
        logL[i] = log2_ceil(full[i] ? 3 * M[i] - 1 : 2 * M[i] - 1);
        loff[i + 1] = loff[i] + (int64_t(1) << logL[i]);
        maxN = std::max(maxN, N[i]);
    }
    b->sumN = b->noff[P]; b->sumM = b->moff[P]; b->sumG = goff[P]; b->sumL = loff[P];
    // member plans and their arena
    std::vector<size_t> pos(P + 1, 0);
    b->plans.resize(P);
    for (int64_t i = 0; i < P; ++i) {
        Plan* p = new Plan();
        p->device = b->device;
        p->sms = b->sms;
        p->M = M[i]; p->N = N[i]; p->Ms = 2 * M[i]; p->m = m; p->kernel = kernel; p->sigma = sigma; p->tau = tau;
        p->ansatz = INFFT_ANSATZ_OVERDETERMINED;
        p->logMs = log2_ceil(p->Ms);
        p->nnz_cap = N[i] * (2 * (int64_t)m + 1);
        p->batch_member = true;
        b->plans[i] = p;
        Carver c;
        plan_layout(p, c, true);
        pos[i + 1] = pos[i] + ((c.off + 255) & ~(size_t)255);
    }
    cudaError_t e = cudaMalloc(&b->arena, pos[P]);
    for (int64_t i = 0; i < P && e == cudaSuccess; ++i) {
        Carver c;
        c.base = (char*)b->arena + pos[i];
        plan_layout(b->plans[i], c, true);
    }
    auto alloc = [&](auto** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc((void**)ptr, bytes + 16);
    };
    alloc(&b->x_all, b->sumN * sizeof(double));
    alloc(&b->g_all, b->sumG * sizeof(float2));
    alloc(&b->bhat, b->sumL * sizeof(float2));
    alloc(&b->tw, TW_N * sizeof(float2));
    alloc(&b->stage_f, b->sumN * sizeof(float2));
    alloc(&b->stage_fhat, b->sumM * sizeof(float2));
    alloc(&b->probs, P * sizeof(BatchProblem));
    alloc(&b->huge_probs, P * huge_problem_bytes());
    alloc(&b->job_off, (P + 1) * sizeof(int32_t));
    alloc(&b->order, P * sizeof(int32_t));
    alloc(&b->ticket, sizeof(int32_t));
    alloc(&b->pat_args, P * sizeof(PatternArgs));
    alloc(&b->tier_args, P * tier_args_bytes());
    alloc(&b->pat_order, P * sizeof(int32_t));
    alloc(&b->tier_tile_off, (P + 1) * sizeof(int32_t));
    alloc(&b->tier_work, 5 * (P + 1) * sizeof(int32_t));
    alloc(&b->d_counters, P * sizeof(void*));
    alloc(&b->d_col_off, P * sizeof(void*));
    alloc(&b->d_J, P * sizeof(void*));
    alloc(&b->d_Ms, P * sizeof(int32_t));
    alloc(&b->d_info, 8 * P * sizeof(double));
    // blocked solver for columns above the warp tier: one scratch triangle per CTA,
    // sized for the largest column a problem can have (at most N nodes)
    b->huge_nmax = (int)std::min<int64_t>(maxN, HUGE_NMAX);
    b->huge_slots = maxN > LSQ_WARP2_NMAX ? b->sms : 0;
    if (b->huge_slots) {
        alloc(&b->huge_scratch, huge_scratch_doubles(b->huge_slots, b->huge_nmax) * sizeof(double));
        alloc(&b->job_order, b->sumG * sizeof(int32_t));
        alloc(&b->job_work, (HUGE_NMAX + 8) * sizeof(int32_t));
    }
    // tiles of the batched spreading: at most one per cols grid points plus one per
    // wblk weights of the largest possible nnz (the buffer for the smallest shape; the
    // apply launches the bound of the batch's shape)
    for (int sh = 0; sh < TILE_SHAPE_COUNT; ++sh) {
        const int cols = 1 << TILE_SHAPES[sh].log_cols, wblk = 1 << TILE_SHAPES[sh].log_wblk;
        for (int64_t i = 0; i < P; ++i)
            b->shape_tiles[sh] += (2 * M[i] + cols - 1) / cols + b->plans[i]->nnz_cap / wblk + 1;
        b->max_tiles = std::max(b->max_tiles, b->shape_tiles[sh]);
    }
    alloc(&b->tiles, 2 * b->max_tiles * sizeof(int4));
    alloc(&b->tile_count, P * sizeof(int32_t));
    alloc(&b->tile_off, (P + 1) * sizeof(int32_t));
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_err(e, "allocate batch");
    }
    // descriptors and tables (host-built, copied once)
    std::vector<BatchProblem> hp(P);
    std::vector<const int32_t*> hc(P), ho(P);
    std::vector<const double*> hj(P);
    std::vector<int32_t> hms(P);
    for (int64_t i = 0; i < P; ++i) {
        Plan* p = b->plans[i];
        p->x = b->x_all + b->noff[i];
        BatchProblem& d = hp[i];
        d.w32 = p->w32; d.w64 = p->w64; d.wlo = p->wlo; d.wide = p->wide; d.perm = p->perm;
        d.col_start = p->col_start; d.col_count = p->col_count; d.col_off = p->col_off;
        d.bhat = b->bhat + loff[i];
        d.f_off = b->noff[i]; d.fhat_off = b->moff[i]; d.g_off = goff[i];
        d.N = (int)N[i]; d.M = (int)M[i]; d.logL = logL[i]; d.sym = kernel == INFFT_KERNEL_SYM;
        d.full = full[i];
        hc[i] = p->counters; ho[i] = p->col_off; hj[i] = p->J; hms[i] = (int32_t)p->Ms;
    }
    std::vector<char> hh(P * huge_problem_bytes());
    huge_problems_fill(b->plans.data(), (int)P, hh.data());
    // batch-wide pattern and solver tiers: descriptors, order and tile prefix
    std::vector<PatternArgs> hpat(P);
    std::vector<int32_t> htoff(P + 1, 0), pord(P);
    for (int64_t i = 0; i < P; ++i) {
        Plan* p = b->plans[i];
        PatternArgs& a = hpat[i];
        a.x = p->x; a.xs = p->xs; a.phase = p->phase; a.skey = p->skey; a.perm = p->perm; a.bucket = p->bucket;
        a.cursor = p->cursor; a.seg_list = p->seg_list; a.sort_tmp = p->sort_tmp; a.col_start = p->col_start;
        a.col_count = p->col_count; a.col_off = p->col_off; a.counters = p->counters;
        a.N = (int)p->N; a.Ms = (int)p->Ms; a.m = p->m; a.M = (double)p->M;
        htoff[i + 1] = htoff[i] + (int32_t)((p->Ms + 31) / 32);
    }
    b->total_tiles32 = htoff[P];
    std::iota(pord.begin(), pord.end(), 0);
    std::stable_sort(pord.begin(), pord.end(), [&](int32_t a, int32_t c) { return N[a] + 2 * M[a] > N[c] + 2 * M[c]; });
    std::vector<char> htier(P * tier_args_bytes());
    tier_args_fill(b->plans.data(), (int)P, htier.data());
    std::vector<int32_t> ord(P);
    std::iota(ord.begin(), ord.end(), 0);
    // largest first: grid reads plus transform work (2 or 4 transforms of length L)
    auto cost = [&](int32_t i) { return (double)N[i] + (full[i] ? 2.0 : 4.0) * (double)(int64_t(1) << logL[i]) * logL[i] / 8.0; };
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t c) { return cost(a) > cost(c); });
    std::vector<float2> htw(TW_N);
    for (int t = 0; t < TW_N; ++t) {
        // e^{-2 pi i t/TW_N} from the exactly reduced fraction t/TW_N
        const double a = -2.0 * M_PI * (double)t / (double)TW_N;
        htw[t] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    std::vector<int64_t> hloff(loff.begin(), loff.end() - 1);
    int64_t* d_loff = nullptr;
    e = cudaMemcpy(b->probs, hp.data(), P * sizeof(BatchProblem), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->huge_probs, hh.data(), hh.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->order, ord.data(), P * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->tw, htw.data(), TW_N * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->pat_args, hpat.data(), P * sizeof(PatternArgs), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->tier_args, htier.data(), htier.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->pat_order, pord.data(), P * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->tier_tile_off, htoff.data(), (P + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_counters, hc.data(), P * sizeof(void*), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_col_off, ho.data(), P * sizeof(void*), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_J, hj.data(), P * sizeof(void*), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_Ms, hms.data(), P * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&d_loff, P * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemcpy(d_loff, hloff.data(), P * sizeof(int64_t), cudaMemcpyHostToDevice);
    // every member's counters start at zero
    for (int64_t i = 0; i < P && e == cudaSuccess; ++i)
        e = cudaMemsetAsync(b->plans[i]->counters, 0, CNT_N * sizeof(int32_t), 0);
    if (e == cudaSuccess) e = phase_table_init();
    const size_t chirp_smem = (size_t)pad16(TW_N) * sizeof(float2);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_chirp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chirp_smem);
    if (e == cudaSuccess) {
        k_batch_chirp<<<(unsigned)P, BATCH_FFT_THREADS, chirp_smem>>>(b->probs, b->bhat, d_loff, b->tw);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (d_loff) cudaFree(d_loff);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_err(e, "initialise batch");
    }
    *out = b;
    return INFFT_OK;
}

infft_status infft_batch_set_nodes(infft_batch_t b, const double* x, infft_stream_t stream) {
    if (!b) return set_error(INFFT_EINVAL, "batch is NULL");
    if (!x) return set_error(INFFT_EINVAL, "x is NULL");
    DevGuard g(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    b->last_stream = s;
    cudaError_t e;
    if (on_device(x)) {
        e = cudaMemcpyAsync(b->x_all, x, b->sumN * sizeof(double), cudaMemcpyDeviceToDevice, s);
    } else {
        const int64_t j = first_bad_coordinate(x, b->sumN);
        if (j >= 0) return set_error(INFFT_EINVAL, "node x[%lld] = %.17g is not in [-1/2, 1/2)", (long long)j, x[j]);
        e = cudaMemcpyAsync(b->x_all, x, b->sumN * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    if (e != cudaSuccess) return cuda_err(e, "copy nodes");
    b->precomputed = 0;
    // every problem's pattern in one launch (a CTA per problem)
    if ((e = run_pattern_batch(b->pat_args, b->pat_order, (int)b->P, b->sms, s)) != cudaSuccess)
        return cuda_err(e, "pattern");
    for (int64_t i = 0; i < b->P; ++i) b->plans[i]->nodes_set = 1;
    b->nodes_set = 1;
    return INFFT_OK;
}

infft_status infft_batch_precompute(infft_batch_t b, infft_stream_t stream) {
    if (!b) return set_error(INFFT_EINVAL, "batch is NULL");
    if (!b->nodes_set) return set_error(INFFT_ENOTREADY, "infft_batch_precompute before infft_batch_set_nodes");
    DevGuard g(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    b->last_stream = s;
    cudaError_t e;
    // every problem's columns up to 64 nodes: one launch per solver tier over all problems
    if ((e = run_precompute_batch(b->tier_args, (int)b->P, b->tier_tile_off, (int)b->total_tiles32, b->tier_work,
                                  b->sms, s)) != cudaSuccess)
        return cuda_err(e, "precompute");
    for (int64_t i = 0; i < b->P; ++i) b->plans[i]->precomputed = 1;
    if (b->huge_slots &&
        (e = run_precompute_huge(b->huge_probs, (int)b->P, b->job_off, b->job_order, b->job_work, b->huge_scratch,
                                 b->huge_slots, b->huge_nmax, s)) !=
            cudaSuccess)
        return cuda_err(e, "large-column precompute");
    if ((e = build_tiles(b, s)) != cudaSuccess) return cuda_err(e, "spreading tiles");
    b->precomputed = 1;
    return INFFT_OK;
}

namespace {

// The two launches of the batched apply on device buffers.
cudaError_t run_batch_apply(infft_batch_t b, const float2* fin, float2* fout, cudaStream_t s) {
    cudaError_t e;
    if ((e = launch_batch_spread(b->tile_shape, (unsigned)b->shape_tiles[b->tile_shape], b->probs, b->tiles,
                                 b->tile_off + b->P, fin,
                                 b->g_all, s)) != cudaSuccess)
        return e;
    const size_t smem = (size_t)(pad16(TW_N) + BATCH_MMAX) * sizeof(float2);
    if ((e = cudaFuncSetAttribute(k_batch_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(b->ticket, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    k_batch_fft<<<b->sms, BATCH_FFT_THREADS, smem, s>>>(b->probs, (int)b->P, b->order, b->g_all, fout, b->tw,
                                                        b->ticket);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace

int32_t infft_batch_tile_shape_count(void) { return TILE_SHAPE_COUNT; }

infft_status infft_batch_tile_shape(int32_t id, int32_t* cols, int32_t* weights) {
    if (id < 0 || id >= TILE_SHAPE_COUNT)
        return set_error(INFFT_EINVAL, "tile shape id %d not in [0, %d)", id, TILE_SHAPE_COUNT);
    if (cols) *cols = 1 << TILE_SHAPES[id].log_cols;
    if (weights) *weights = 1 << TILE_SHAPES[id].log_wblk;
    return INFFT_OK;
}

int32_t infft_batch_get_tile_shape(infft_batch_t b) { return b ? b->tile_shape : -1; }

infft_status infft_batch_set_tile_shape(infft_batch_t b, int32_t id, infft_stream_t stream) {
    if (!b) return set_error(INFFT_EINVAL, "batch is NULL");
    if (id == -1) id = TILE_SHAPE_DEFAULT;
    if (id < 0 || id >= TILE_SHAPE_COUNT)
        return set_error(INFFT_EINVAL, "tile shape id %d not in [-1, %d)", id, TILE_SHAPE_COUNT);
    b->tile_shape = id;
    if (!b->precomputed) return INFFT_OK;   // the precompute cuts the tiles
    DevGuard g(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    b->last_stream = s;
    cudaError_t e = build_tiles(b, s);
    if (e != cudaSuccess) return cuda_err(e, "spreading tiles");
    return INFFT_OK;
}

infft_status infft_batch_tune_apply(infft_batch_t b, int32_t repeats, float* ms_out, int32_t* best,
                                    infft_stream_t stream) {
    if (!b) return set_error(INFFT_EINVAL, "batch is NULL");
    if (repeats < 1 || repeats > 10000) return set_error(INFFT_EINVAL, "repeats must be in [1, 10000] (got %d)", repeats);
    if (!b->precomputed) return set_error(INFFT_ENOTREADY, "infft_batch_tune_apply before infft_batch_precompute");
    DevGuard g(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    b->last_stream = s;
    cudaEvent_t ea = nullptr, eb = nullptr;
    cudaError_t e = cudaEventCreate(&ea);
    if (e == cudaSuccess) e = cudaEventCreate(&eb);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->stage_f, 0, b->sumN * sizeof(float2), s);
    const int keep = b->tile_shape;
    int best_id = -1;
    float best_ms = 0.f;
    for (int id = 0; id < TILE_SHAPE_COUNT && e == cudaSuccess; ++id) {
        b->tile_shape = id;
        e = build_tiles(b, s);
        for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = run_batch_apply(b, b->stage_f, b->stage_fhat, s);
        if (e == cudaSuccess) e = cudaEventRecord(ea, s);
        for (int r = 0; r < repeats && e == cudaSuccess; ++r) e = run_batch_apply(b, b->stage_f, b->stage_fhat, s);
        if (e == cudaSuccess) e = cudaEventRecord(eb, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(eb);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ea, eb);
        ms /= (float)repeats;
        if (ms_out) ms_out[id] = ms;
        if (e == cudaSuccess && (best_id < 0 || ms < best_ms)) {
            best_id = id;
            best_ms = ms;
        }
    }
    if (ea) cudaEventDestroy(ea);
    if (eb) cudaEventDestroy(eb);
    b->tile_shape = e == cudaSuccess ? best_id : keep;
    const cudaError_t e2 = build_tiles(b, s);
    if (e != cudaSuccess) return cuda_err(e, "tune batched apply");
    if (e2 != cudaSuccess) return cuda_err(e2, "spreading tiles");
    if (best) *best = best_id;
    return INFFT_OK;
}

infft_status infft_batch_apply(infft_batch_t b, const float* f, float* fhat, infft_stream_t stream) {
    if (!b) return set_error(INFFT_EINVAL, "batch is NULL");
    if (!f || !fhat) return set_error(INFFT_EINVAL, "f and fhat must not be NULL");
    if (!b->precomputed) return set_error(INFFT_ENOTREADY, "infft_batch_apply before infft_batch_precompute");
    DevGuard g(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    b->last_stream = s;
    cudaError_t e;
    const float2* fin = (const float2*)f;
    if (!on_device(f)) {
        if ((e = cudaMemcpyAsync(b->stage_f, f, b->sumN * sizeof(float2), cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_err(e, "copy f to device");
        fin = b->stage_f;
    }
    const bool host_out = !on_device(fhat);
    float2* fout = host_out ? b->stage_fhat : (float2*)fhat;
    if ((e = run_batch_apply(b, fin, fout, s)) != cudaSuccess) return cuda_err(e, "apply");
    if (host_out) {
        if ((e = cudaMemcpyAsync(fhat, b->stage_fhat, b->sumM * sizeof(float2), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
            return cuda_err(e, "copy fhat to host");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_err(e, "synchronize");
    }
    return INFFT_OK;
}

infft_status infft_batch_get_info(infft_batch_t b, infft_batch_info* info) {
    if (!b || !info) return set_error(INFFT_EINVAL, "batch and info must not be NULL");
    DevGuard g(b->device);
    cudaError_t e = cudaStreamSynchronize(b->last_stream);
    if (e != cudaSuccess) return cuda_err(e, "synchronize");
    std::memset(info, 0, sizeof *info);
    info->P = b->P; info->sum_N = b->sumN; info->sum_M = b->sumM; info->m = b->m;
    info->nodes_set = b->nodes_set; info->precomputed = b->precomputed;
    if (!b->nodes_set) return INFFT_OK;
    k_batch_info<<<(unsigned)b->P, 256>>>(b->d_counters, b->d_col_off, b->d_J, b->d_Ms, b->d_info);
    count_launches(1);
    std::vector<double> h(8 * b->P);
    if ((e = cudaMemcpy(h.data(), b->d_info, h.size() * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_err(e, "read batch info");
    for (int64_t i = 0; i < b->P; ++i) {
        const double* o = &h[8 * i];
        info->nnz += (int64_t)o[0];
        info->max_column = std::max(info->max_column, (int32_t)o[1]);
        info->empty_columns += (int64_t)o[2];
        info->bad_nodes += (int64_t)o[3];
        if (b->precomputed) {
            info->fallback_columns += (int64_t)o[4];
            info->unsupported_columns += (int64_t)o[5];
            info->objective += o[6];
            info->large_columns += (int64_t)o[7];
        }
    }
    return INFFT_OK;
}

infft_status infft_batch_copy_problem(infft_batch_t b, int64_t i, int32_t* perm, int32_t* col_start,
                                      int32_t* col_count, int32_t* col_offset, double* weights, double* objective) {
    if (!b) return set_error(INFFT_EINVAL, "batch is NULL");
    if (i < 0 || i >= b->P) return set_error(INFFT_EINVAL, "problem %lld out of range", (long long)i);
    Plan* p = b->plans[i];
    p->last_stream = b->last_stream;
    return infft_copy_plan_data(p, perm, col_start, col_count, col_offset, weights, objective);
}

infft_status infft_batch_destroy(infft_batch_t b) {
    if (!b) return INFFT_OK;
    {
        DevGuard g(b->device);
        cudaDeviceSynchronize();
        batch_free(b);
    }
    return INFFT_OK;
}

}  // extern "C"
