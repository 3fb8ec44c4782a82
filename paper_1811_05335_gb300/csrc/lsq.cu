// Precomputation of B_opt (Sec. 3.2.2, eq:opt_ansatz2 .. eq:solution_ansatz2).
//
// For every grid point l the real coefficients b_l on I(l) minimise
// ||L_l b - e_l||^2 + mu ||b||^2, L_l = F D H_l (eq:matrix_Ll) with the Dirichlet
// choice (Remark remark:Dirichlet_ansatz2).  Because F^* F = M_sigma I_M, the
// normal matrix has the closed form Re G_{jj'} = Re kappa(x_j - x_j') and the
// right-hand side Re r_j = Re kappa(l/M_sigma - x_j), where
//   full: Re kappa(t) = cos(pi t) sin(pi M t) / (M_sigma sin(pi t)),
//   sym : Re kappa(t) = sin(pi (M-1) t) / (M_sigma sin(pi t))   (eq:kernel_Dirichlet)
//                     = full - cos(pi M t) / M_sigma.
// mu = tau * Re kappa(0) (Tikhonov; the paper assumes full rank).  The systems
// are solved in fp64 by Cholesky with reciprocal pivots; a failed pivot retries
// with mu * 1e3 (twice) and is counted as a fallback column.
//
// GB300 executes fp64 at 1/64 of the fp32 rate, so the kernels are organised to
// minimise fp64 warp instructions:
//   * thread tier: one THREAD per column (tiles whose largest |I(l)| is <= 17), a
//     private packed triangle in shared memory (lane-interleaved), Gram entries
//     shared across the 32 columns of a warp tile;
//   * group tiers: G lanes per column (tiles whose largest |I(l)| is <= 25, 33, 48
//     or 64; the last two in sub-tiles of 16 and 8 columns), Gram entries shared
//     across the (sub-)tile;
//   * warp tier: one warp per column, lanes own rows (|I(l)| <= 64, columns of tiles
//     holding a larger one);
//   * CTA tier: one CTA per column (|I(l)| <= 224), packed triangle; in a batch, the
//     blocked solver in four parts by column size instead (k_lsq_huge).
// Columns too large for a tier go to a device-side work list for the next one.
//
// The kernel values and the thread tier's register Cholesky are in lsq_device.cuh.
#include <algorithm>
#include <cstring>

#include "lsq_device.cuh"

namespace {

constexpr int TILE_UMAX = 128;   // largest union of nodes a warp tile shares in shared memory

template <int NMAX> constexpr int tri_doubles() { return NMAX * (NMAX + 1) / 2; }
template <int NMAX> constexpr size_t tile_warp_bytes() {
    return (size_t)32 * tri_doubles<NMAX>() * sizeof(double) + (size_t)TILE_UMAX * 3 * sizeof(double) +
           (64 + 2 * TILE_UMAX) * sizeof(int);
}

// Writes Re G_l + mu I (lower triangle) of one column into its private triangle T
// (stride 32), evaluating every entry itself.
INFFT_D void fill_gram(double* T, const double* __restrict__ xs, const double2* __restrict__ ph, int s, int n,
                       int N, double mu, const KernelParams& kp) {
    int qi = s;
    for (int i = 0; i < n; ++i) {
        const double xi = xs[qi];
        const double2 pi = ph[qi];
        int qj = s;
        for (int j = 0; j < i; ++j) {
            T[(trow(i) + j) * 32] = re_kappa(xi, xs[qj], pi, ph[qj], kp);
            if (++qj == N) qj = 0;
        }
        T[(trow(i) + i) * 32] = kp.diag + mu;
        if (++qi == N) qi = 0;
    }
}

// One thread per column; a warp owns a tile of 32 consecutive columns.  The first
// tier visits every tile and routes those whose largest column exceeds its NMAX to
// the tile lists of the larger thread tiers, or their columns to the warp tier.  Shared memory
// per warp: each lane's packed lower triangle, lane-interleaved (element e of lane
// t at [e * 32 + t]) so the 32 threads never collide on a bank, plus the tile's
// union of nodes.  Consecutive columns share most of their nodes (I(l) and
// I(l+1) are overlapping ranges of sorted nodes), so the lanes evaluate each node
// pair of the union once and scatter the value into the triangle of every column
// that contains both nodes; a tile whose union does not fit falls back to
// per-column evaluation.
template <int NMAX, int WARPS, bool BATCH = false>
__global__ void __launch_bounds__(WARPS * 32)
k_lsq_thread(const double* __restrict__ xs_, const double2* __restrict__ ph_, const int32_t* __restrict__ col_start_,
             const int32_t* __restrict__ col_count_, const int32_t* __restrict__ col_off_, int N_, int Ms_,
             KernelParams kp_, double mu0_, double* __restrict__ w64_, float* __restrict__ w32_,
             double* __restrict__ Jout_, uint8_t* __restrict__ wide_, const int32_t* __restrict__ tiles_in,
             int tiles_counter, int32_t* __restrict__ route_mid_, int32_t* __restrict__ route_big_,
             int32_t* __restrict__ route_48_, int32_t* __restrict__ route_64_,
             int32_t* __restrict__ col_list_, int32_t* __restrict__ counters_, TierBatch tb) {
    extern __shared__ double lsq_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* wbase = (double*)((char*)lsq_smem + (size_t)wid * tile_warp_bytes<NMAX>());
    double* T = wbase + lane;                                   // T[e * 32]
    double* ux = wbase + 32 * tri_doubles<NMAX>();              // union x      [TILE_UMAX]
    double2* up = (double2*)(ux + TILE_UMAX);                   // union phases [TILE_UMAX]
    int* crs = (int*)(up + TILE_UMAX);                          // tile-relative start per lane [32]
    int* cnn = crs + 32;                                        // size per lane [32]
    int* cfst = cnn + 32;                                       // per union node: first candidate column
    int* clst = cfst + TILE_UMAX;                               // per union node: last candidate column

    // tiles_in == nullptr: every tile, one per warp, routing the tiles this tier cannot
    // take; otherwise the tiles of the list (persistent warps).  Batch mode (BATCH, routing
    // only): the tiles of all problems, numbered by the prefix tb.off.
    const int ntiles = BATCH ? tb.off[tb.P] : tiles_in ? counters_[tiles_counter] : (Ms_ + 31) / 32;
    const int first = blockIdx.x * WARPS + wid, stride = tiles_in ? gridDim.x * WARPS : ntiles;
    for (int it = first; it < ntiles; it += stride) {
    __syncwarp();
    const int pb = BATCH ? batch_problem(tb.off, tb.P, it) : 0;
    const TierArgs* pa = BATCH ? tb.probs + pb : nullptr;
    const double* __restrict__ xs = BATCH ? pa->xs : xs_;
    const double2* __restrict__ ph = BATCH ? pa->ph : ph_;
    const int32_t* __restrict__ col_start = BATCH ? pa->col_start : col_start_;
    const int32_t* __restrict__ col_count = BATCH ? pa->col_count : col_count_;
    const int32_t* __restrict__ col_off = BATCH ? pa->col_off : col_off_;
    const int N = BATCH ? pa->N : N_, Ms = BATCH ? pa->Ms : Ms_;
    const KernelParams& kp = BATCH ? pa->kp : kp_;
    const double mu0 = BATCH ? pa->mu0 : mu0_;
    double* __restrict__ w64 = BATCH ? pa->w64 : w64_;
    float* __restrict__ w32 = BATCH ? pa->w32 : w32_;
    double* __restrict__ Jout = BATCH ? pa->J : Jout_;
    uint8_t* __restrict__ wide = BATCH ? pa->wide : wide_;
    int32_t* __restrict__ route_mid = BATCH ? pa->tiles_mid : route_mid_;
    int32_t* __restrict__ route_big = BATCH ? pa->tiles_big : route_big_;
    int32_t* __restrict__ route_48 = BATCH ? pa->tiles_48 : route_48_;
    int32_t* __restrict__ route_64 = BATCH ? pa->tiles_64 : route_64_;
    // in a batch, the columns of tiles above 64 nodes go straight to the big list, which the
    // blocked solver takes (its smallest part has eight CTAs per SM); alone, to the warp tier
    int32_t* __restrict__ col_list = BATCH ? pa->big_list : col_list_;
    int32_t* __restrict__ counters = BATCH ? pa->counters : counters_;
    const int tile = BATCH ? it - tb.off[pb] : tiles_in ? tiles_in[it] : it;
    const int p = tile * 32 + lane;
    const bool live = p < Ms;
    const int n = live ? col_count[p] : 0;
    int D = n;
    for (int o = 16; o; o >>= 1) D = max(D, __shfl_xor_sync(0xffffffffu, D, o));
    if (D > NMAX) {                        // only the routing tier meets such tiles
        if (D <= LSQ_THREAD_NMAX2) {
            if (lane == 0) route_mid[atomicAdd(&counters[CNT_TILES_MID], 1)] = tile;
        } else if (D <= LSQ_THREAD_NMAX3) {
            if (lane == 0) route_big[atomicAdd(&counters[CNT_TILES_BIG], 1)] = tile;
        } else if (D <= LSQ_GROUP_NMAX4) {
            if (lane == 0) route_48[atomicAdd(&counters[CNT_TILES_48], 1)] = tile;
        } else if (D <= LSQ_WARP2_NMAX) {
            if (lane == 0) route_64[atomicAdd(&counters[CNT_TILES_64], 1)] = tile;
        } else if (n > 0) {
            col_list[atomicAdd(&counters[BATCH ? CNT_BIG_LIST : CNT_LIST_A], 1)] = p;
        } else if (live) {                 // empty columns of a tile sent to the warp tier end here
            Jout[p] = 1.0;
            wide[p] = 0;
        }
        continue;
    }
    const int s = live ? col_start[p] : 0;
    const int S = __shfl_sync(0xffffffffu, s, 0);
    int rs = s - S;
    if (rs < 0) rs += N;
    const bool mine = n > 0;
    // the union of the tile's ranges, in tile-relative positions [0, U)
    int U = mine ? rs + n : 0;
    const bool fits = !mine || (rs + n <= TILE_UMAX);
    for (int o = 16; o; o >>= 1) U = max(U, __shfl_xor_sync(0xffffffffu, U, o));
    const bool tile_ok = __all_sync(0xffffffffu, fits) && U <= N && U > 0;

    const double tl = col_t(p, Ms);
    const double2 pl = phase_of(kp.M, tl);
    double v[NMAX];
    if (tile_ok) {
        crs[lane] = mine ? rs : 0;
        cnn[lane] = n;
        for (int q = lane; q < U; q += 32) {
            int g = S + q;
            if (g >= N) g -= N;
            ux[q] = xs[g];
            up[q] = ph[g];
        }
        __syncwarp();
        for (int q = lane; q < U; q += 32) {
            int cf = 32, cl = -1;
            for (int c = 0; c < 32; ++c) {
                if (cnn[c] > 0 && crs[c] + cnn[c] > q && cf == 32) cf = c;
                if (cnn[c] > 0 && crs[c] <= q) cl = c;
            }
            cfst[q] = cf;
            clst[q] = cl;
        }
        // the near path needs the union and the columns' grid points to lie within
        // 1/64 of each other without crossing the seam
        const double x0 = ux[0], x1 = ux[U - 1];
        const bool near = !kp.sym && x1 >= x0 && x1 - x0 <= 1.0 / 64.0 &&
                          __all_sync(0xffffffffu, !mine || (tl >= x0 - 1.0 / 64.0 && tl <= x1 + 1.0 / 64.0));
        __syncwarp();
        // every pair (a, b), a < b < a + D, of the union, evaluated once
        const int per = D - 1;
        if (per > 0) {
            const int pairs = U * per;
            const int qa = 32 / per, ra = 32 % per;
            int a = lane / per, off = lane % per;
            for (int e = lane; e < pairs; e += 32) {
                const int b = a + 1 + off;
                if (b < U) {
                    const int c0 = cfst[b], c1 = clst[a];
                    if (c0 <= c1) {
                        const double val = near ? kappa_near(ux[b] - ux[a], up[b], up[a], kp)
                                                : re_kappa(ux[b], ux[a], up[b], up[a], kp);
                        for (int c = c0; c <= c1; ++c) {
                            const int r0 = crs[c];
                            if (r0 <= a && b < r0 + cnn[c]) wbase[(trow(b - r0) + (a - r0)) * 32 + c] = val;
                        }
                    }
                }
                a += qa;
                off += ra;
                if (off >= per) { off -= per; ++a; }
            }
        }
        if (mine) {
#pragma unroll
            for (int i = 0; i < NMAX; ++i) {
                if (i < n) {
                    v[i] = near ? kappa_near(tl - ux[rs + i], pl, up[rs + i], kp)
                                : re_kappa(tl, ux[rs + i], pl, up[rs + i], kp);
                    T[(trow(i) + i) * 32] = kp.diag + mu0;
                }
            }
        }
        __syncwarp();
    } else if (mine) {
        fill_gram(T, xs, ph, s, n, N, mu0, kp);
        int q = s;
#pragma unroll
        for (int i = 0; i < NMAX; ++i) {
            if (i < n) {
                v[i] = re_kappa(tl, xs[q], pl, ph[q], kp);
                if (++q == N) q = 0;
            }
        }
    }
    if (!mine) {
        if (live) { Jout[p] = 1.0; wide[p] = 0; }
        continue;
    }
    const int off = col_off[p];
    double mu = mu0, ysq = 0.0;
    bool ok = chol_solve<NMAX>(T, n, v, ysq);
    for (int attempt = 1; attempt < 3 && !ok; ++attempt) {
        mu *= 1e3;
        fill_gram(T, xs, ph, s, n, N, mu, kp);
        int q = s;
#pragma unroll
        for (int i = 0; i < NMAX; ++i) {
            if (i < n) {
                v[i] = re_kappa(tl, xs[q], pl, ph[q], kp);
                if (++q == N) q = 0;
            }
        }
        ok = chol_solve<NMAX>(T, n, v, ysq);
    }
    if (!ok) {
        for (int i = 0; i < n; ++i) { w64[off + i] = 0.0; w32[off + i] = 0.0f; }
        Jout[p] = 1.0;
        wide[p] = 0;
        atomicAdd(&counters[CNT_FALLBACK], 1);
        continue;
    }
    if (mu != mu0) atomicAdd(&counters[CNT_FALLBACK], 1);
    double bsq = 0.0, babs = 0.0;
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        if (i < n) {
            store_b(w64, w32, kp.wlo, off + i, v[i]);
            bsq = fma(v[i], v[i], bsq);
            babs += fabs(v[i]);
        }
    }
    // J_l = ||L b - e_l||^2 = 1 - r.b - mu ||b||^2 at the regularised optimum
    Jout[p] = 1.0 - ysq - mu * bsq;
    wide[p] = babs > WIDE_COLUMN_L1;
    }
}

// ---------------------------------------------------------------- tiers 2/3: G lanes per column

// A CTA of G warps owns a tile of 32 consecutive columns; G lanes share a column.
// Thread-per-column triangles of |I(l)| = 25 or 33 leave room for one or two warps
// per SM, which cannot keep the SM's fp64 pipes busy; with G lanes per column the
// same shared memory serves G times as many warps.  The factorisation is
// row-distributed and left-looking: for each pivot column j a lane forms the
// entries of the rows it owns from row j (a broadcast within the group), the
// pivot reaches the group by a shuffle, and no cross-lane sum is needed.  r is
// stored as an extra last row (index NMAX), so its elimination is the forward
// solve y = L^{-1} r.  The loops run to the warp's largest column Dw; columns of a
// warp smaller than Dw are padded with identity rows, which leave their solution
// unchanged, and rows Dw .. NMAX - 1 stay out of the system.  Lane g owns rows
// NMAX - g - G t (slots t = 0, 1, ...), counted from the bottom: rows finished early
// sit in the high slots, which drop out of the loop as j passes them, so few issued
// multiply-adds fall on finished rows, and which lane and slot hold a row is known
// at compile time.
// A CTA may also take its 32-column tile as 32 / TC sub-tiles of TC columns (TC = 16 and 8 for
// the 48- and 64-node tiers, whose triangles of 32 columns would not fit shared memory); the
// triangles of a sub-tile are interleaved with element stride TC + 1.

template <int NMAX> constexpr int aug_doubles() { return (NMAX + 1) * (NMAX + 2) / 2; }
// the triangles' region rounded up to 16 bytes, so that the double2 phases after it are aligned
template <int NMAX, int TC = 32> constexpr int group_tri_doubles() { return (aug_doubles<NMAX>() * (TC + 1) + 1) & ~1; }
template <int NMAX, int TC = 32> constexpr size_t group_smem_bytes() {
    return (size_t)group_tri_doubles<NMAX, TC>() * sizeof(double) + (size_t)TILE_UMAX * 3 * sizeof(double) +
           (size_t)(64 + 2 * TILE_UMAX + 8) * sizeof(int);
}

// 1/sqrt(d) of a Cholesky pivot, and whether d is a positive number inside the fp32
// normal range (otherwise the pivot counts as failed).  d is rounded to fp32 by
// integer operations, the hardware fp32 reciprocal square root gives r with relative
// error below 2^-21, and one Newton step with its second-order term,
// r (1 - e)^{-1/2} ~ r (1 + e/2 + 3 e^2 / 8) with e = 1 - d r^2, leaves an error of
// order 3 (e/2)^3 < 2^-60: below fp64 rounding.
INFFT_D double rsqrt_pivot(double d, bool& ok) {
    const long long bits = __double_as_longlong(d);
    const int hi = (int)(bits >> 32);
    const int ex = hi >> 20;                       // biased exponent (the sign is bit 31 of hi)
    ok = hi > 0 && ex >= 1023 - 126 && ex <= 1023 + 127;
    const int fb = ((ex - 1023 + 127) << 23) | ((hi & 0xfffff) << 3) | (int)((unsigned long long)bits >> 29 & 7);
    const float rf = rsqrtf(__int_as_float(ok ? fb : 0x3f800000));
    const int rb = __float_as_int(rf);
    const int rhi = ((((rb >> 23) & 0xff) - 127 + 1023) << 20) | ((rb & 0x7fffff) >> 3);
    double r = __hiloint2double(rhi, (int)((unsigned)rb << 29));
    const double h = d * r;
    const double e = fma(-h, r, 1.0);
    const double t = fma(e, 0.375, 0.5);
    return fma(r * e, t, r);
}

// Left-looking Cholesky of the augmented triangle (rows 0 .. Dw - 1 and the r row NMAX)
// of one column, G lanes per column.  rowo[t]: element offset of row NMAX - g - G t
// (row 0 where that is negative).  Rows of L overwrite the matrix, reciprocal pivots
// the diagonal.  Returns false on a failed pivot (the same on all lanes of a group).
template <int NMAX, int G, int R, int GS>
INFFT_D bool group_factor(double* Tc, int g, int gbase, int Dw, const int (&rowo)[R]) {
    bool ok = true;
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
        if (j < Dw) {
            double acc[R];
#pragma unroll
            for (int t = 0; t < R; ++t)
                if (NMAX - G * t >= j) acc[t] = Tc[rowo[t] + j * GS];   // slot holds rows >= j
#pragma unroll
            for (int k = 0; k < j; ++k) {
                const double ljk = Tc[(trow(j) + k) * GS];
#pragma unroll
                for (int t = 0; t < R; ++t)
                    if (NMAX - G * t >= j) acc[t] = fma(-Tc[rowo[t] + k * GS], ljk, acc[t]);
            }
            // row j: lane (NMAX - j) % G, slot (NMAX - j) / G
            const double dj = __shfl_sync(0xffffffffu, acc[(NMAX - j) / G], gbase + (NMAX - j) % G);
            bool okj;
            const double rp = rsqrt_pivot(dj, okj);
            ok = ok && okj;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                if (NMAX - G * t >= j) {
                    const int i = NMAX - g - G * t;
                    if (i > j) Tc[rowo[t] + j * GS] = acc[t] * rp;
                }
            }
            if (g == (NMAX - j) % G) Tc[(trow(j) + j) * GS] = rp;
            __syncwarp();
        }
    }
    return ok;
}

// Backward solve L^T b = y by columns of L^T: bacc[t] holds y of row NMAX - g - G t
// on entry and b on exit; colo[t] = max(NMAX - g - G t, 0) * GS.
template <int NMAX, int G, int R, int GS>
INFFT_D void group_backsolve(const double* Tc, int g, int gbase, int Dw, const int (&colo)[R], double (&bacc)[R]) {
#pragma unroll
    for (int i = NMAX - 1; i >= 0; --i) {
        if (i < Dw) {
            const double rp = Tc[(trow(i) + i) * GS];
            const int ti = (NMAX - i) / G, gi = (NMAX - i) % G;
            const double bi = __shfl_sync(0xffffffffu, bacc[ti] * rp, gbase + gi);
            if (g == gi) bacc[ti] = bi;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                if (NMAX - G * t - (G - 1) < i) {                        // slot holds rows < i
                    const int k = NMAX - g - G * t;
                    if (k < i && k >= 0) bacc[t] = fma(-Tc[trow(i) * GS + colo[t]], bi, bacc[t]);
                }
            }
        }
    }
}

// A column's augmented system evaluated directly from the sorted nodes (tiles whose
// union does not fit, and retries with a larger mu), rows and r entries split over
// the G lanes: Re G_l + mu I for rows < n, identity rows for n <= i < Dw, r in row NMAX.
template <int NMAX, int G, int GS>
INFFT_D void group_fill_direct(double* Tc, int g, int n, int Dw, int s, const double* __restrict__ xs,
                               const double2* __restrict__ ph, int N, double tl, double2 pl, double mu,
                               const KernelParams& kp) {
    for (int i = g; i < Dw; i += G) {
        if (i < n) {
            int qi = s + i;
            if (qi >= N) qi -= N;
            const double xi = xs[qi];
            const double2 pi = ph[qi];
            int qk = s;
            for (int k = 0; k < i; ++k) {
                Tc[(trow(i) + k) * GS] = re_kappa(xi, xs[qk], pi, ph[qk], kp);
                if (++qk == N) qk = 0;
            }
            Tc[(trow(i) + i) * GS] = kp.diag + mu;
        } else {
            for (int k = 0; k < i; ++k) Tc[(trow(i) + k) * GS] = 0.0;
            Tc[(trow(i) + i) * GS] = 1.0;
        }
    }
    for (int k = g; k < Dw; k += G) {
        double r = 0.0;
        if (k < n) {
            int q = s + k;
            if (q >= N) q -= N;
            r = re_kappa(tl, xs[q], pl, ph[q], kp);
        }
        Tc[(trow(NMAX) + k) * GS] = r;
    }
}

template <int NMAX, int G, bool BATCH = false, int TC = 32>
__global__ void __launch_bounds__(TC * G, 1)
k_lsq_group(const double* __restrict__ xs_, const double2* __restrict__ ph_, const int32_t* __restrict__ col_start_,
            const int32_t* __restrict__ col_count_, const int32_t* __restrict__ col_off_, int N_, int Ms_,
            KernelParams kp_, double mu0_, double* __restrict__ w64_, float* __restrict__ w32_,
            double* __restrict__ Jout_, uint8_t* __restrict__ wide_, const int32_t* __restrict__ tiles_,
            int tiles_counter, int32_t* __restrict__ counters_, TierBatch tb) {
    constexpr int C = 32 / G;          // columns per warp
    constexpr int R = (NMAX + G) / G;  // row slots per lane: rows 0 .. NMAX, from the bottom
    constexpr int NT = TC * G;         // threads per CTA
    constexpr int GS = TC + 1;         // element stride of the interleaved triangles
    static_assert(32 % G == 0 && 32 % TC == 0 && NT % 32 == 0, "G and TC divide the warp; whole warps");
    static_assert(group_tri_doubles<NMAX, TC>() % 2 == 0 && TILE_UMAX % 2 == 0, "double2 phases 16-byte aligned");
    extern __shared__ double lsq_smem[];
    double* T = lsq_smem;                                       // element e of column c at T[e * GS + c]
    double* ux = T + group_tri_doubles<NMAX, TC>();             // union x      [TILE_UMAX]
    double2* up = (double2*)(ux + TILE_UMAX);                   // union phases [TILE_UMAX]
    int* crs = (int*)(up + TILE_UMAX);                          // tile-relative start per column [32]
    int* cnn = crs + 32;                                        // size per column [32]
    int* cfst = cnn + 32;                                       // per union node: first candidate column
    int* clst = cfst + TILE_UMAX;                               // per union node: last candidate column
    int* tinfo = clst + TILE_UMAX;                              // S, U, D, tile_ok, near

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane % G, gbase = lane - g;
    const int c = wid * C + lane / G;
    double* Tc = T + c;
    int rowo[R], colo[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
        const int i = max(NMAX - g - G * t, 0);
        rowo[t] = trow(i) * GS;
        colo[t] = i * GS;
    }

    // batch mode (BATCH): the listed tiles of all problems, numbered by the prefix tb.off
    const int ntiles = BATCH ? tb.off[tb.P] : counters_[tiles_counter];
    for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
        __syncthreads();                  // the previous tile is done with shared memory
        const int pb = BATCH ? batch_problem(tb.off, tb.P, it) : 0;
        const TierArgs* pa = BATCH ? tb.probs + pb : nullptr;
        const double* __restrict__ xs = BATCH ? pa->xs : xs_;
        const double2* __restrict__ ph = BATCH ? pa->ph : ph_;
        const int32_t* __restrict__ col_start = BATCH ? pa->col_start : col_start_;
        const int32_t* __restrict__ col_count = BATCH ? pa->col_count : col_count_;
        const int32_t* __restrict__ col_off = BATCH ? pa->col_off : col_off_;
        const int N = BATCH ? pa->N : N_, Ms = BATCH ? pa->Ms : Ms_;
        const KernelParams& kp = BATCH ? pa->kp : kp_;
        const double mu0 = BATCH ? pa->mu0 : mu0_;
        double* __restrict__ w64 = BATCH ? pa->w64 : w64_;
        float* __restrict__ w32 = BATCH ? pa->w32 : w32_;
        double* __restrict__ Jout = BATCH ? pa->J : Jout_;
        uint8_t* __restrict__ wide = BATCH ? pa->wide : wide_;
        int32_t* __restrict__ counters = BATCH ? pa->counters : counters_;
        const int32_t* __restrict__ tiles =
            BATCH ? (tiles_counter == CNT_TILES_MID ? pa->tiles_mid
                     : tiles_counter == CNT_TILES_BIG ? pa->tiles_big
                     : tiles_counter == CNT_TILES_48 ? pa->tiles_48 : pa->tiles_64) : tiles_;
        const int tile = tiles[BATCH ? it - tb.off[pb] : it];
        for (int sub = 0; sub < 32 / TC; ++sub) {
        const int cb = tile * 32 + sub * TC;   // the sub-tile's first column
        if (cb >= Ms) break;                   // uniform over the CTA
        __syncthreads();                       // the previous sub-tile is done with shared memory
        if (wid == 0) {
            const int p = cb + lane;
            const bool live = lane < TC && p < Ms;
            const int n = live ? col_count[p] : 0;
            const int s = live ? col_start[p] : 0;
            const int S = __shfl_sync(0xffffffffu, s, 0);
            int rs = s - S;
            if (rs < 0) rs += N;
            const bool mine = n > 0;
            int U = mine ? rs + n : 0, D = n;
            const bool fits = !mine || (rs + n <= TILE_UMAX);
            for (int o = 16; o; o >>= 1) {
                U = max(U, __shfl_xor_sync(0xffffffffu, U, o));
                D = max(D, __shfl_xor_sync(0xffffffffu, D, o));
            }
            const bool tile_ok = __all_sync(0xffffffffu, fits) && U <= N && U > 0;
            crs[lane] = mine ? rs : 0;
            cnn[lane] = n;
            if (lane == 0) {
                tinfo[0] = S;
                tinfo[1] = U;
                tinfo[2] = D;
                tinfo[3] = tile_ok;
            }
        }
        __syncthreads();
        const int S = tinfo[0], U = tinfo[1], D = tinfo[2];
        const bool tile_ok = tinfo[3] != 0;
        if (D > NMAX) {                   // not routed here; kept as a guard
            if (threadIdx.x == 0) atomicAdd(&counters[CNT_UNSUPPORTED], 1);
            continue;
        }
        const int p = cb + c;
        const bool live = p < Ms;
        const int n = cnn[c], rs = crs[c];
        const double tl = col_t(p, Ms);
        const double2 pl = phase_of(kp.M, tl);
        bool near = false;
        if (tile_ok) {
            for (int q = threadIdx.x; q < U; q += NT) {
                int gq = S + q;
                if (gq >= N) gq -= N;
                ux[q] = xs[gq];
                up[q] = ph[gq];
            }
            __syncthreads();
            for (int q = threadIdx.x; q < U; q += NT) {
                int cf = TC, cl = -1;
                for (int cc = 0; cc < TC; ++cc) {
                    if (cnn[cc] > 0 && crs[cc] + cnn[cc] > q && cf == TC) cf = cc;
                    if (cnn[cc] > 0 && crs[cc] <= q) cl = cc;
                }
                cfst[q] = cf;
                clst[q] = cl;
            }
            if (wid == 0) {
                // the near path needs the union and the columns' grid points to lie
                // within 1/64 of each other without crossing the seam
                const double x0 = ux[0], x1 = ux[U - 1];
                const double tq = col_t(cb + lane, Ms);
                const bool mine = cnn[lane] > 0;
                const bool nr = !kp.sym && x1 >= x0 && x1 - x0 <= 1.0 / 64.0 &&
                                __all_sync(0xffffffffu, !mine || (tq >= x0 - 1.0 / 64.0 && tq <= x1 + 1.0 / 64.0));
                if (lane == 0) tinfo[4] = nr;
            }
            __syncthreads();
            near = tinfo[4] != 0;
            // every pair (a, b), a < b < a + D, of the union, evaluated once
            const int per = D - 1;
            if (per > 0) {
                const int pairs = U * per;
                const int qa = NT / per, ra = NT % per;
                int a = threadIdx.x / per, off = threadIdx.x % per;
                for (int e = threadIdx.x; e < pairs; e += NT) {
                    const int b = a + 1 + off;
                    if (b < U) {
                        const int c0 = cfst[b], c1 = clst[a];
                        if (c0 <= c1) {
                            const double val = near ? kappa_near(ux[b] - ux[a], up[b], up[a], kp)
                                                    : re_kappa(ux[b], ux[a], up[b], up[a], kp);
                            for (int cc = c0; cc <= c1; ++cc) {
                                const int r0 = crs[cc];
                                if (r0 <= a && b < r0 + cnn[cc]) T[(trow(b - r0) + (a - r0)) * GS + cc] = val;
                            }
                        }
                    }
                    a += qa;
                    off += ra;
                    if (off >= per) { off -= per; ++a; }
                }
            }
            __syncthreads();
        }
        // this warp's largest column: the extent of the (padded) systems
        int Dw = n;
        for (int o = 16; o; o >>= 1) Dw = max(Dw, __shfl_xor_sync(0xffffffffu, Dw, o));
        if (live && n == 0 && g == 0) {
            Jout[p] = 1.0;
            wide[p] = 0;
        }
        const int s = live ? col_start[p] : 0;
        double mu = mu0;

        if (tile_ok) {
            for (int i = g; i < Dw; i += G) {
                if (i < n) {
                    Tc[(trow(i) + i) * GS] = kp.diag + mu;
                } else {
                    for (int k = 0; k < i; ++k) Tc[(trow(i) + k) * GS] = 0.0;
                    Tc[(trow(i) + i) * GS] = 1.0;
                }
            }
            for (int k = g; k < Dw; k += G) {
                double r = 0.0;
                if (k < n)
                    r = near ? kappa_near(tl - ux[rs + k], pl, up[rs + k], kp)
                             : re_kappa(tl, ux[rs + k], pl, up[rs + k], kp);
                Tc[(trow(NMAX) + k) * GS] = r;
            }
        } else {
            group_fill_direct<NMAX, G, GS>(Tc, g, n, Dw, s, xs, ph, N, tl, pl, mu, kp);
        }
        bool need = n > 0;
        const int off = live ? col_off[p] : 0;
        for (int attempt = 0; attempt < 3; ++attempt) {
            if (attempt > 0) {
                if (!__any_sync(0xffffffffu, need)) break;
                if (need) {
                    mu *= 1e3;
                    group_fill_direct<NMAX, G, GS>(Tc, g, n, Dw, s, xs, ph, N, tl, pl, mu, kp);
                }
            }
            __syncwarp();
            const bool ok = group_factor<NMAX, G, R, GS>(Tc, g, gbase, Dw, rowo);
            double bacc[R], ysq = 0.0;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                bacc[t] = Tc[trow(NMAX) * GS + colo[t]];
                const int k = NMAX - g - G * t;
                if (k >= 0 && k < n) ysq = fma(bacc[t], bacc[t], ysq);
            }
            group_backsolve<NMAX, G, R, GS>(Tc, g, gbase, Dw, colo, bacc);
            const bool write = need && ok;
            double bsq = 0.0, babs = 0.0;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int k = NMAX - g - G * t;
                if (write && k >= 0 && k < n) {
                    store_b(w64, w32, kp.wlo, off + k, bacc[t]);
                    bsq = fma(bacc[t], bacc[t], bsq);
                    babs += fabs(bacc[t]);
                }
            }
#pragma unroll
            for (int o = G / 2; o; o >>= 1) {
                ysq += __shfl_xor_sync(0xffffffffu, ysq, o);
                bsq += __shfl_xor_sync(0xffffffffu, bsq, o);
                babs += __shfl_xor_sync(0xffffffffu, babs, o);
            }
            if (write && g == 0) {
                // J_l = ||L b - e_l||^2 = 1 - r.b - mu ||b||^2 at the regularised optimum
                Jout[p] = 1.0 - ysq - mu * bsq;
                wide[p] = babs > WIDE_COLUMN_L1;
                if (mu != mu0) atomicAdd(&counters[CNT_FALLBACK], 1);
            }
            if (write) need = false;
        }
        if (need) {
            for (int k = g; k < n; k += G) { w64[off + k] = 0.0; w32[off + k] = 0.0f; }
            if (g == 0) {
                Jout[p] = 1.0;
                wide[p] = 0;
                atomicAdd(&counters[CNT_FALLBACK], 1);
            }
        }
        }   // sub-tiles
    }
}

// ---------------------------------------------------------------- tier 4: warp per column

// One warp per column; lane t owns rows t, t + 32, ... (NMAX / 32 rows).  Columns
// come from `list` (count at counters[list_counter]).
template <int NMAX, int WARPS, bool BATCH = false>
__global__ void __launch_bounds__(WARPS * 32)
k_lsq_warp(const double* __restrict__ xs_, const double2* __restrict__ ph_, const int32_t* __restrict__ col_start_,
           const int32_t* __restrict__ col_count_, const int32_t* __restrict__ col_off_, int N_, int Ms_,
           KernelParams kp_, double mu0_, double* __restrict__ w64_, float* __restrict__ w32_,
           double* __restrict__ Jout_, uint8_t* __restrict__ wide_, const int32_t* __restrict__ list_,
           int list_counter, int32_t* __restrict__ next_list_, int next_counter, int32_t* __restrict__ counters_,
           TierBatch tb) {
    constexpr int ROWS = NMAX / 32;
    constexpr int LD = NMAX + 1;     // padded row stride: conflict-free column access
    extern __shared__ double lsq_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* A = lsq_smem + (size_t)wid * (NMAX * LD + 4 * NMAX);
    double* r = A + NMAX * LD;
    double* xl = r + NMAX;
    double2* pv = (double2*)(xl + NMAX);
    // batch mode (BATCH): the listed columns of all problems, numbered by the prefix tb.off
    const int total = BATCH ? tb.off[tb.P] : counters_[list_counter];
    for (int it = blockIdx.x * WARPS + wid; it < total; it += gridDim.x * WARPS) {
        const int pb = BATCH ? batch_problem(tb.off, tb.P, it) : 0;
        const TierArgs* pa = BATCH ? tb.probs + pb : nullptr;
        const double* __restrict__ xs = BATCH ? pa->xs : xs_;
        const double2* __restrict__ ph = BATCH ? pa->ph : ph_;
        const int32_t* __restrict__ col_start = BATCH ? pa->col_start : col_start_;
        const int32_t* __restrict__ col_count = BATCH ? pa->col_count : col_count_;
        const int32_t* __restrict__ col_off = BATCH ? pa->col_off : col_off_;
        const int N = BATCH ? pa->N : N_, Ms = BATCH ? pa->Ms : Ms_;
        const KernelParams& kp = BATCH ? pa->kp : kp_;
        const double mu0 = BATCH ? pa->mu0 : mu0_;
        double* __restrict__ w64 = BATCH ? pa->w64 : w64_;
        float* __restrict__ w32 = BATCH ? pa->w32 : w32_;
        double* __restrict__ Jout = BATCH ? pa->J : Jout_;
        uint8_t* __restrict__ wide = BATCH ? pa->wide : wide_;
        int32_t* __restrict__ counters = BATCH ? pa->counters : counters_;
        int32_t* __restrict__ next_list = BATCH ? pa->big_list : next_list_;
        const int32_t* __restrict__ list = BATCH ? pa->list_a : list_;
        const int p = list[BATCH ? it - tb.off[pb] : it];
        const int n = col_count[p];
        if (n > NMAX) {
            if (lane == 0) next_list[atomicAdd(&counters[next_counter], 1)] = p;
            continue;
        }
        const int s = col_start[p], off = col_off[p];
        const double tl = col_t(p, Ms);
        const double2 pl = phase_of(kp.M, tl);
        for (int i = lane; i < n; i += 32) {
            int q = s + i;
            if (q >= N) q -= N;
            xl[i] = xs[q];
            pv[i] = ph[q];
        }
        __syncwarp();
        const int ntri = n * (n + 1) / 2;
        double mu = mu0;
        bool ok = false;
        for (int attempt = 0; attempt < 3 && !ok; ++attempt) {
            for (int i = lane; i < n; i += 32) r[i] = re_kappa(tl, xl[i], pl, pv[i], kp);
            for (int e = lane; e < ntri; e += 32) {
                int i, j;
                tri_index(e, i, j);
                A[i * LD + j] = (i == j) ? kp.diag + mu : re_kappa(xl[i], xl[j], pv[i], pv[j], kp);
            }
            __syncwarp();
            ok = true;
            for (int k = 0; k < n; ++k) {
                const double akk = A[k * LD + k];
                if (!(akk > 0.0) || !isfinite(akk)) { ok = false; break; }   // warp-uniform
                const double rp = rsqrt(akk);
                double lik[ROWS];
#pragma unroll
                for (int t = 0; t < ROWS; ++t) {
                    const int i = lane + 32 * t;
                    lik[t] = (i > k && i < n) ? A[i * LD + k] * rp : 0.0;
                }
                __syncwarp();
#pragma unroll
                for (int t = 0; t < ROWS; ++t) {
                    const int i = lane + 32 * t;
                    if (i > k && i < n) A[i * LD + k] = lik[t];
                }
                if (lane == (k & 31)) A[k * LD + k] = rp;
                __syncwarp();
#pragma unroll
                for (int t = 0; t < ROWS; ++t) {
                    const int i = lane + 32 * t;
                    if (i > k && i < n)
                        for (int j = k + 1; j <= i; ++j) A[i * LD + j] = fma(-lik[t], A[j * LD + k], A[i * LD + j]);
                }
                __syncwarp();
            }
            if (!ok) mu *= 1e3;
        }
        if (!ok) {
            for (int i = lane; i < n; i += 32) { w64[off + i] = 0.0; w32[off + i] = 0.0f; }
            if (lane == 0) { Jout[p] = 1.0; wide[p] = 0; atomicAdd(&counters[CNT_FALLBACK], 1); }
            __syncwarp();
            continue;
        }
        if (lane == 0 && mu != mu0) atomicAdd(&counters[CNT_FALLBACK], 1);
        // forward: y = L^{-1} r (r overwritten by y); ||y||^2 = r . b
        double ysq = 0.0;
        for (int k = 0; k < n; ++k) {
            const double yk = r[k] * A[k * LD + k];
            ysq = fma(yk, yk, ysq);
            __syncwarp();
            if (lane == (k & 31)) r[k] = yk;
#pragma unroll
            for (int t = 0; t < ROWS; ++t) {
                const int i = lane + 32 * t;
                if (i > k && i < n) r[i] = fma(-A[i * LD + k], yk, r[i]);
            }
            __syncwarp();
        }
        // backward: L^T b = y (r overwritten by b)
        for (int k = n - 1; k >= 0; --k) {
            const double bk = r[k] * A[k * LD + k];
            __syncwarp();
            if (lane == (k & 31)) r[k] = bk;
#pragma unroll
            for (int t = 0; t < ROWS; ++t) {
                const int i = lane + 32 * t;
                if (i < k) r[i] = fma(-A[k * LD + i], bk, r[i]);
            }
            __syncwarp();
        }
        double bsq = 0.0, babs = 0.0;
        for (int i = lane; i < n; i += 32) {
            const double b = r[i];
            store_b(w64, w32, kp.wlo, off + i, b);
            bsq = fma(b, b, bsq);
            babs += fabs(b);
        }
        for (int o = 16; o; o >>= 1) {
            bsq += __shfl_xor_sync(0xffffffffu, bsq, o);
            babs += __shfl_xor_sync(0xffffffffu, babs, o);
        }
        if (lane == 0) {
            Jout[p] = 1.0 - ysq - mu * bsq;
            wide[p] = babs > WIDE_COLUMN_L1;
        }
        __syncwarp();
    }
}

template <int NMAX, int WARPS> constexpr size_t warp_smem_bytes() {
    return (size_t)WARPS * (NMAX * (NMAX + 1) + 4 * NMAX) * sizeof(double);
}

// ---------------------------------------------------------------- tier 4: CTA per column

constexpr int CTA_THREADS = 256;
constexpr int CN = LSQ_CTA_NMAX;

__global__ void __launch_bounds__(CTA_THREADS)
k_lsq_cta(const double* __restrict__ xs, const double2* __restrict__ ph, const int32_t* __restrict__ col_start,
          const int32_t* __restrict__ col_count, const int32_t* __restrict__ col_off, int N, int Ms,
          KernelParams kp, double mu0, double* __restrict__ w64, float* __restrict__ w32,
          double* __restrict__ Jout, uint8_t* __restrict__ wide, const int32_t* __restrict__ big_list,
          int32_t* __restrict__ counters) {
    extern __shared__ double smem[];
    double* A = smem;                  // CN (CN + 1) / 2, packed rows
    double* r = A + CN * (CN + 1) / 2; // CN
    double* xl = r + CN;               // CN
    double2* pv = (double2*)(xl + CN); // CN
    __shared__ int s_ok;
    __shared__ double s_red[2 * (CTA_THREADS / 32)];
    const int total = counters[CNT_BIG_LIST];   // filled by the warp tiers
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int p = big_list[it];
        const int n = col_count[p], s = col_start[p], off = col_off[p];
        if (n > CN) {
            for (int i = threadIdx.x; i < n; i += CTA_THREADS) { w64[off + i] = 0.0; w32[off + i] = 0.0f; }
            if (threadIdx.x == 0) { Jout[p] = 1.0; wide[p] = 0; atomicAdd(&counters[CNT_UNSUPPORTED], 1); }
            continue;
        }
        const double tl = col_t(p, Ms);
        const double2 pl = phase_of(kp.M, tl);
        for (int i = threadIdx.x; i < n; i += CTA_THREADS) {
            int q = s + i;
            if (q >= N) q -= N;
            xl[i] = xs[q];
            pv[i] = ph[q];
        }
        __syncthreads();
        const int ntri = n * (n + 1) / 2;
        double mu = mu0;
        bool ok = false;
        for (int attempt = 0; attempt < 3 && !ok; ++attempt) {
            for (int i = threadIdx.x; i < n; i += CTA_THREADS) r[i] = re_kappa(tl, xl[i], pl, pv[i], kp);
            for (int e = threadIdx.x; e < ntri; e += CTA_THREADS) {
                int i, j;
                tri_index(e, i, j);
                A[trow(i) + j] = (i == j) ? kp.diag + mu : re_kappa(xl[i], xl[j], pv[i], pv[j], kp);
            }
            if (threadIdx.x == 0) s_ok = 1;
            __syncthreads();
            for (int k = 0; k < n; ++k) {
                const double akk = A[trow(k) + k];
                if (!(akk > 0.0) || !isfinite(akk)) {   // block-uniform
                    if (threadIdx.x == 0) s_ok = 0;
                    break;
                }
                const double rp = rsqrt(akk);
                __syncthreads();
                for (int i = k + 1 + threadIdx.x; i < n; i += CTA_THREADS) A[trow(i) + k] *= rp;
                if (threadIdx.x == 0) A[trow(k) + k] = rp;
                __syncthreads();
                const int m2 = n - k - 1;
                const int nt = m2 * (m2 + 1) / 2;
                for (int e = threadIdx.x; e < nt; e += CTA_THREADS) {
                    int a, b;
                    tri_index(e, a, b);
                    const int i = k + 1 + a, j = k + 1 + b;
                    A[trow(i) + j] = fma(-A[trow(i) + k], A[trow(j) + k], A[trow(i) + j]);
                }
                __syncthreads();
            }
            __syncthreads();
            ok = s_ok != 0;
            if (!ok) mu *= 1e3;
            __syncthreads();
        }
        if (!ok) {
            for (int i = threadIdx.x; i < n; i += CTA_THREADS) { w64[off + i] = 0.0; w32[off + i] = 0.0f; }
            if (threadIdx.x == 0) { Jout[p] = 1.0; wide[p] = 0; atomicAdd(&counters[CNT_FALLBACK], 1); }
            __syncthreads();
            continue;
        }
        if (threadIdx.x == 0 && mu != mu0) atomicAdd(&counters[CNT_FALLBACK], 1);
        double ysq = 0.0;
        for (int k = 0; k < n; ++k) {
            const double yk = r[k] * A[trow(k) + k];
            ysq = fma(yk, yk, ysq);
            __syncthreads();
            if (threadIdx.x == 0) r[k] = yk;
            for (int i = k + 1 + threadIdx.x; i < n; i += CTA_THREADS) r[i] = fma(-A[trow(i) + k], yk, r[i]);
            __syncthreads();
        }
        for (int k = n - 1; k >= 0; --k) {
            const double bk = r[k] * A[trow(k) + k];
            __syncthreads();
            if (threadIdx.x == 0) r[k] = bk;
            for (int i = threadIdx.x; i < k; i += CTA_THREADS) r[i] = fma(-A[trow(k) + i], bk, r[i]);
            __syncthreads();
        }
        double bsq = 0.0, babs = 0.0;
        for (int i = threadIdx.x; i < n; i += CTA_THREADS) {
            const double b = r[i];
            store_b(w64, w32, kp.wlo, off + i, b);
            bsq = fma(b, b, bsq);
            babs += fabs(b);
        }
        for (int o = 16; o; o >>= 1) {
            bsq += __shfl_xor_sync(0xffffffffu, bsq, o);
            babs += __shfl_xor_sync(0xffffffffu, babs, o);
        }
        if ((threadIdx.x & 31) == 0) {
            s_red[threadIdx.x >> 5] = bsq;
            s_red[CTA_THREADS / 32 + (threadIdx.x >> 5)] = babs;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0, a = 0.0;
            for (int w = 0; w < CTA_THREADS / 32; ++w) { t += s_red[w]; a += s_red[CTA_THREADS / 32 + w]; }
            Jout[p] = 1.0 - ysq - mu * t;
            wide[p] = a > WIDE_COLUMN_L1;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- tier 5: large columns
//
// Columns above the warp tier of the problems of a batch (clustered nodes put
// tens to hundreds of nodes into the columns next to the cluster) are solved in
// one launch, one CTA per column with the packed triangle in a global scratch
// slot of the CTA.  Blocked right-looking Cholesky:
// a panel of HUGE_PB columns is staged in shared memory, factored there, written
// back, and the trailing triangle is updated in 4x4 register blocks (fp64-pipe
// bound: 256 multiply-adds per 32 global accesses).  The kernel serves every
// problem of a batch: jobs are numbered across the problems' big lists through
// an exclusive prefix of their lengths.

constexpr int HUGE_PB = 16;
constexpr int HUGE_PS = HUGE_PB + 1;   // panel row stride: rows 4 apart hit different banks
// the blocked solver's parts: largest column of each (panel capacity), threads and CTAs per SM
constexpr int HUGE_PARTS = 4;
constexpr int HUGE_PART_LIMIT[HUGE_PARTS] = {HUGE_NMAX, 512, 256, 128};
constexpr int HUGE_PART_THREADS[HUGE_PARTS] = {256, 256, 128, 64};
constexpr int HUGE_PART_MINB[HUGE_PARTS] = {1, 2, 4, 8};

__global__ void k_huge_prefix(const HugeProblem* __restrict__ probs, int P, int32_t* __restrict__ job_off) {
    __shared__ int32_t part[1024];
    // one CTA of 1024 threads: per-thread serial sums, then a shared scan
    const int per = (P + 1023) / 1024;
    const int a = threadIdx.x * per, b = min(a + per, P);
    int32_t sum = 0;
    for (int i = a; i < b; ++i) sum += probs[i].counters[CNT_BIG_LIST];
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
        job_off[i] = run;
        run += probs[i].counters[CNT_BIG_LIST];
    }
    if (threadIdx.x == 1023) job_off[P] = part[1023];
}

// Largest-first order of the jobs (a counting sort by column size, descending):
// the cost of a column grows as n^3, so taking the largest first keeps the CTAs
// of the persistent solver evenly loaded.
INFFT_D int job_size(const HugeProblem* __restrict__ probs, int P, const int32_t* __restrict__ job_off, int job,
                     int nmax) {
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (job_off[mid] <= job) lo = mid; else hi = mid - 1;
    }
    const HugeProblem& pr = probs[lo];
    return min(pr.col_count[pr.big_list[job - job_off[lo]]], nmax);
}

__global__ void k_job_hist(const HugeProblem* __restrict__ probs, int P, const int32_t* __restrict__ job_off,
                           int nmax, int32_t* __restrict__ hist) {
    const int total = job_off[P];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += gridDim.x * blockDim.x)
        atomicAdd(&hist[nmax - job_size(probs, P, job_off, j, nmax)], 1);
}

// exclusive prefix of the nmax + 1 bucket counts (one CTA of 1024 threads), in place
__global__ void __launch_bounds__(1024) k_job_scan(int32_t* __restrict__ hist, int nb) {
    __shared__ int32_t part[1024];
    const int per = (nb + 1023) / 1024;
    const int a = threadIdx.x * per, b = min(a + per, nb);
    int32_t sum = 0;
    for (int i = a; i < b; ++i) sum += hist[i];
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
        const int32_t c = hist[i];
        hist[i] = run;
        run += c;
    }
}

__global__ void k_job_scatter(const HugeProblem* __restrict__ probs, int P, const int32_t* __restrict__ job_off,
                              int nmax, int32_t* __restrict__ cursor, int32_t* __restrict__ order) {
    const int total = job_off[P];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += gridDim.x * blockDim.x)
        order[atomicAdd(&cursor[nmax - job_size(probs, P, job_off, j, nmax)], 1)] = j;
}

// The jobs are solved in four parts of the largest-first order, each by its own
// launch: columns above 512 nodes (panel capacity 1024 rows, one CTA of 256 threads per
// SM), 257 .. 512 nodes (two CTAs per SM), 129 .. 256 nodes (four CTAs of 128 threads)
// and up to 128 nodes (eight CTAs of 64 threads): smaller columns need less shared
// memory, and more CTAs per SM overlap their latency-bound panel, fill and back-solve
// steps.  split[k]: the number of jobs above HUGE_PART_LIMIT[k + 1] nodes; after
// k_job_scatter each bucket's cursor holds its end.
__global__ void k_job_split(const int32_t* __restrict__ cursor, int nmax, int32_t* __restrict__ split) {
    constexpr int L1 = HUGE_PART_LIMIT[1], L2 = HUGE_PART_LIMIT[2], L3 = HUGE_PART_LIMIT[3];
    split[0] = nmax > L1 ? cursor[nmax - L1 - 1] : 0;
    split[1] = nmax > L2 ? cursor[nmax - L2 - 1] : 0;
    split[2] = nmax > L3 ? cursor[nmax - L3 - 1] : 0;
}

template <int PMAX, int NTH, int MINB>
__global__ void __launch_bounds__(NTH, MINB)
k_lsq_huge(const HugeProblem* __restrict__ probs, int P, const int32_t* __restrict__ job_off,
           const int32_t* __restrict__ order, int32_t* __restrict__ ticket, const int32_t* __restrict__ split,
           int part, double* __restrict__ scratch, size_t slot_doubles, int nmax) {
    extern __shared__ double smem[];
    double* pan = smem;                          // PMAX x HUGE_PB panel (row stride HUGE_PS)
    double* r = pan + PMAX * HUGE_PS;            // PMAX
    double* xl = r + PMAX;                       // PMAX
    double2* pv = (double2*)(xl + PMAX);         // PMAX
    __shared__ double s_red[2 * (NTH / 32)];
    __shared__ double s_y[HUGE_PB];              // b of the current block of rows (back solve)
    __shared__ int s_t;
    double* A = scratch + (size_t)blockIdx.x * slot_doubles;
    const int first = part == 0 ? 0 : split[part - 1];
    const int last = part == HUGE_PARTS - 1 ? job_off[P] : split[part];
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_t = first + atomicAdd(ticket, 1);
        __syncthreads();
        const int t = s_t;
        __syncthreads();
        if (t >= last) break;
        const int job = order[t];   // largest columns first
        int lo = 0, hi = P - 1;   // problem: the last i with job_off[i] <= job
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (job_off[mid] <= job) lo = mid; else hi = mid - 1;
        }
        const HugeProblem& pr = probs[lo];
        const int p = pr.big_list[job - job_off[lo]];
        const int n = pr.col_count[p], s = pr.col_start[p], off = pr.col_off[p], N = pr.N;
        if (tid == 0 && n > LSQ_CTA_NMAX) atomicAdd(&pr.counters[CNT_HUGE_LIST], 1);
        if (n > nmax) {
            for (int i = tid; i < n; i += NTH) { pr.w64[off + i] = 0.0; pr.w32[off + i] = 0.0f; }
            if (tid == 0) { pr.J[p] = 1.0; pr.wide[p] = 0; atomicAdd(&pr.counters[CNT_UNSUPPORTED], 1); }
            continue;
        }
        const KernelParams& kp = pr.kp;
        const double tl = col_t(p, pr.Ms);
        const double2 pl = phase_of(kp.M, tl);
        for (int i = tid; i < n; i += NTH) {
            int q = s + i;
            if (q >= N) q -= N;
            xl[i] = pr.xs[q];
            pv[i] = pr.ph[q];
        }
        __syncthreads();
        double mu = pr.mu;
        double ysq = 0.0;
        bool ok = false;
        for (int attempt = 0; attempt < 3 && !ok; ++attempt) {
            for (int i = tid; i < n; i += NTH) r[i] = re_kappa(tl, xl[i], pl, pv[i], kp);
            const int ntri = n * (n + 1) / 2;
            for (int e = tid; e < ntri; e += NTH) {   // packed row-major: entry e is (i, j)
                int i, j;
                tri_index(e, i, j);
                A[e] = (i == j) ? kp.diag + mu : re_kappa(xl[i], xl[j], pv[i], pv[j], kp);
            }
            ysq = 0.0;
            __syncthreads();
            bool failed = false;   // block-uniform: decided on shared values
            for (int kb = 0; kb < n && !failed; kb += HUGE_PB) {
                const int w = min(HUGE_PB, n - kb), R = n - kb;
                for (int e = tid; e < R * HUGE_PB; e += NTH) {
                    const int i = e / HUGE_PB, c = e % HUGE_PB;
                    pan[i * HUGE_PS + c] = (c < w && c <= i) ? A[trow(kb + i) + kb + c] : 0.0;
                }
                __syncthreads();
                for (int c = 0; c < w; ++c) {
                    const double akk = pan[c * HUGE_PS + c];
                    if (!(akk > 0.0) || !isfinite(akk)) {
                        failed = true;
                        break;
                    }
                    const double rp = rsqrt(akk);
                    __syncthreads();
                    for (int i = c + 1 + tid; i < R; i += NTH) pan[i * HUGE_PS + c] *= rp;
                    if (tid == 0) pan[c * HUGE_PS + c] = rp;
                    __syncthreads();
                    // rank-1 update of the panel's remaining columns c' in (c, w), rows i >= c'
                    const int nc = w - c - 1;
                    for (int e = tid; e < (R - c - 1) * nc; e += NTH) {
                        const int i = c + 1 + e / nc, cc = c + 1 + e % nc;
                        if (cc <= i) pan[i * HUGE_PS + cc] = fma(-pan[i * HUGE_PS + c], pan[cc * HUGE_PS + c],
                                                                 pan[i * HUGE_PS + cc]);
                    }
                    __syncthreads();
                }
                if (failed) break;
                // forward solve L y = r for this panel's columns (the column-oriented
                // elimination needs only the panel, which is in shared memory)
                for (int c = 0; c < w; ++c) {
                    const double yc = r[kb + c] * pan[c * HUGE_PS + c];
                    ysq = fma(yc, yc, ysq);
                    __syncthreads();
                    if (tid == 0) r[kb + c] = yc;
                    for (int i = c + 1 + tid; i < R; i += NTH) r[kb + i] = fma(-pan[i * HUGE_PS + c], yc, r[kb + i]);
                    __syncthreads();
                }
                for (int e = tid; e < R * HUGE_PB; e += NTH) {
                    const int i = e / HUGE_PB, c = e % HUGE_PB;
                    if (c < w && c <= i) A[trow(kb + i) + kb + c] = pan[i * HUGE_PS + c];
                }
                // trailing update of rows/columns [kb + w, n) in 4x4 blocks
                const int T = n - kb - w;
                const int nb = (T + 3) >> 2;
                const int nblk = nb * (nb + 1) / 2;
                for (int bk = tid; bk < nblk; bk += NTH) {
                    int bi, bj;
                    tri_index(bk, bi, bj);
                    const int i0 = w + 4 * bi, j0 = w + 4 * bj;   // panel row indices
                    // the block's entries are requested first, so that their latency passes
                    // under the 256 multiply-adds
                    double old[4][4], acc[4][4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int i = kb + i0 + a;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const int j = kb + j0 + b;
                            old[a][b] = (i < n && j <= i) ? A[trow(i) + j] : 0.0;
                            acc[a][b] = 0.0;
                        }
                    }
#pragma unroll 4
                    for (int c = 0; c < HUGE_PB; ++c) {
                        double li[4], lj[4];
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            li[a] = (i0 + a < R) ? pan[(i0 + a) * HUGE_PS + c] : 0.0;
                            lj[a] = (j0 + a < R) ? pan[(j0 + a) * HUGE_PS + c] : 0.0;
                        }
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int b = 0; b < 4; ++b) acc[a][b] = fma(li[a], lj[b], acc[a][b]);
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int i = kb + i0 + a;
                        if (i >= n) break;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const int j = kb + j0 + b;
                            if (j <= i) A[trow(i) + j] = old[a][b] - acc[a][b];
                        }
                    }
                }
                __syncthreads();
            }
            __syncthreads();
            ok = !failed;
            if (!ok) mu *= 1e3;
        }
        if (!ok) {
            for (int i = tid; i < n; i += NTH) { pr.w64[off + i] = 0.0; pr.w32[off + i] = 0.0f; }
            if (tid == 0) { pr.J[p] = 1.0; pr.wide[p] = 0; atomicAdd(&pr.counters[CNT_FALLBACK], 1); }
            __syncthreads();
            continue;
        }
        if (tid == 0 && mu != pr.mu) atomicAdd(&pr.counters[CNT_FALLBACK], 1);
        // back solve L^T b = y in blocks of HUGE_PB rows of L staged in shared memory
        // (row k of L is contiguous in the packed storage; diagonal = reciprocal pivot)
        for (int kb = ((n - 1) / HUGE_PB) * HUGE_PB; kb >= 0; kb -= HUGE_PB) {
            const int hb = min(HUGE_PB, n - kb);
            __syncthreads();
            for (int c = 0; c < hb; ++c)
                for (int i = tid; i <= kb + c; i += NTH) pan[c * PMAX + i] = A[trow(kb + c) + i];
            __syncthreads();
            // the block's own rows by warp 0 (lane c holds y_{kb+c}, then b), b_k for k from
            // the block's last row down; then every row above the block takes the block's b
            // out of r at once (three barriers per block instead of two per row)
            if (tid < 32) {
                double v = tid < hb ? r[kb + tid] : 0.0;
                for (int c = hb - 1; c >= 0; --c) {
                    const double bc = __shfl_sync(0xffffffffu, v, c) * pan[c * PMAX + kb + c];
                    if (tid == c) v = bc;
                    else if (tid < c) v = fma(-pan[c * PMAX + kb + tid], bc, v);
                }
                if (tid < hb) {
                    r[kb + tid] = v;
                    s_y[tid] = v;
                }
            }
            __syncthreads();
            for (int i = tid; i < kb; i += NTH) {
                double acc = r[i];
                for (int c = hb - 1; c >= 0; --c) acc = fma(-pan[c * PMAX + i], s_y[c], acc);
                r[i] = acc;
            }
        }
        __syncthreads();
        double bsq = 0.0, babs = 0.0;
        for (int i = tid; i < n; i += NTH) {
            const double b = r[i];
            store_b(pr.w64, pr.w32, pr.kp.wlo, off + i, b);
            bsq = fma(b, b, bsq);
            babs += fabs(b);
        }
        for (int o = 16; o; o >>= 1) {
            bsq += __shfl_xor_sync(0xffffffffu, bsq, o);
            babs += __shfl_xor_sync(0xffffffffu, babs, o);
        }
        if ((tid & 31) == 0) {
            s_red[tid >> 5] = bsq;
            s_red[NTH / 32 + (tid >> 5)] = babs;
        }
        __syncthreads();
        if (tid == 0) {
            double t = 0.0, a = 0.0;
            for (int w = 0; w < NTH / 32; ++w) { t += s_red[w]; a += s_red[NTH / 32 + w]; }
            pr.J[p] = 1.0 - ysq - mu * t;
            pr.wide[p] = a > WIDE_COLUMN_L1;
        }
        __syncthreads();
    }
}

template <typename K> cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

cudaError_t run_precompute(Plan* p, cudaStream_t s) {
    const int N = (int)p->N, Ms = (int)p->Ms;
    const KernelParams kp = make_kernel_params(p);
    const double mu = p->tau * kp.diag;

    // clear the precompute counters (fallback, unsupported, work lists), keep the pattern's
    cudaError_t e = cudaMemsetAsync(p->counters + CNT_FALLBACK, 0, 2 * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->counters + CNT_LIST_A, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->counters + CNT_BIG_LIST, 0, 3 * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->counters + CNT_HUGE_LIST, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->counters + CNT_TILES_48, 0, 2 * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int sms = p->sms;

    // thread tier: a tile of 32 consecutive columns goes to the first tier whose NMAX
    // covers its largest column (this kernel routes the others); group tiers: G lanes
    // per column; tiles above the last go to the warp tier
    constexpr int A1 = LSQ_THREAD_NMAX1, A2 = LSQ_THREAD_NMAX2, A3 = LSQ_THREAD_NMAX3;
    constexpr int W1 = 5, G2 = LSQ_GROUP_G2, G3 = LSQ_GROUP_G3, W4 = 4;
    auto t1 = k_lsq_thread<A1, W1>;
    auto t2 = k_lsq_group<A2, G2>;
    auto t3 = k_lsq_group<A3, G3>;
    auto t4 = k_lsq_group<LSQ_GROUP_NMAX4, LSQ_GROUP_G4, false, LSQ_GROUP_TC4>;
    auto t5 = k_lsq_group<LSQ_WARP2_NMAX, LSQ_GROUP_G5, false, LSQ_GROUP_TC5>;
    auto k4 = k_lsq_warp<LSQ_WARP2_NMAX, W4>;
    const size_t s1 = W1 * tile_warp_bytes<A1>(), s2 = group_smem_bytes<A2>(), s3 = group_smem_bytes<A3>();
    const size_t st4 = group_smem_bytes<LSQ_GROUP_NMAX4, LSQ_GROUP_TC4>();
    const size_t st5 = group_smem_bytes<LSQ_WARP2_NMAX, LSQ_GROUP_TC5>();
    const size_t s4 = warp_smem_bytes<LSQ_WARP2_NMAX, W4>();
    const size_t s5 = (size_t)(CN * (CN + 1) / 2 + 4 * CN) * sizeof(double);
    if ((e = set_smem(t1, s1)) != cudaSuccess) return e;
    if ((e = set_smem(t2, s2)) != cudaSuccess) return e;
    if ((e = set_smem(t3, s3)) != cudaSuccess) return e;
    if ((e = set_smem(t4, st4)) != cudaSuccess) return e;
    if ((e = set_smem(t5, st5)) != cudaSuccess) return e;
    if ((e = set_smem(k4, s4)) != cudaSuccess) return e;
    if ((e = set_smem(k_lsq_cta, s5)) != cudaSuccess) return e;
    const int tiles = (Ms + 31) / 32;
    int occ2 = 1, occ3 = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, t2, G2 * 32, s2)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ3, t3, G3 * 32, s3)) != cudaSuccess) return e;
    occ2 = std::max(occ2, 1);
    occ3 = std::max(occ3, 1);

    launch_begin(p, "lsq_thread17", s);
    t1<<<(tiles + W1 - 1) / W1, W1 * 32, s1, s>>>(p->xs, p->phase, p->col_start, p->col_count, p->col_off, N, Ms,
                                                  kp, mu, p->w64, p->w32, p->J, p->wide, nullptr, 0, p->tiles_mid,
                                                  p->tiles_big, p->tiles_48, p->tiles_64, p->list_a, p->counters,
                                                  TierBatch{});
    launch_end(p, s);
    launch_begin(p, "lsq_group25", s);
    t2<<<occ2 * sms, G2 * 32, s2, s>>>(p->xs, p->phase, p->col_start, p->col_count, p->col_off, N, Ms, kp, mu,
                                       p->w64, p->w32, p->J, p->wide, p->tiles_mid, CNT_TILES_MID, p->counters,
                                       TierBatch{});
    launch_end(p, s);
    launch_begin(p, "lsq_group33", s);
    t3<<<occ3 * sms, G3 * 32, s3, s>>>(p->xs, p->phase, p->col_start, p->col_count, p->col_off, N, Ms, kp, mu,
                                       p->w64, p->w32, p->J, p->wide, p->tiles_big, CNT_TILES_BIG, p->counters,
                                       TierBatch{});
    launch_end(p, s);
    launch_begin(p, "lsq_group48", s);
    t4<<<sms, LSQ_GROUP_TC4 * LSQ_GROUP_G4, st4, s>>>(p->xs, p->phase, p->col_start, p->col_count, p->col_off, N, Ms,
                                                      kp, mu, p->w64, p->w32, p->J, p->wide, p->tiles_48, CNT_TILES_48,
                                                      p->counters, TierBatch{});
    launch_end(p, s);
    launch_begin(p, "lsq_group64", s);
    t5<<<sms, LSQ_GROUP_TC5 * LSQ_GROUP_G5, st5, s>>>(p->xs, p->phase, p->col_start, p->col_count, p->col_off, N, Ms,
                                                      kp, mu, p->w64, p->w32, p->J, p->wide, p->tiles_64, CNT_TILES_64,
                                                      p->counters, TierBatch{});
    launch_end(p, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // warp tier: columns of tiles whose largest column exceeds the thread tiers, |I(l)| <= 64
    launch_begin(p, "lsq_warp64", s);
    k4<<<2 * sms, W4 * 32, s4, s>>>(p->xs, p->phase, p->col_start, p->col_count, p->col_off, N, Ms, kp, mu,
                                    p->w64, p->w32, p->J, p->wide, p->list_a, CNT_LIST_A, p->big_list,
                                    CNT_BIG_LIST, p->counters, TierBatch{});
    launch_end(p, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // CTA tier: the big list, one CTA per column, |I(l)| <= 224.  Batch members leave
    // their big list to the batch's blocked solver, which takes every problem's list
    // in one launch.
    if (p->batch_member) return cudaGetLastError();
    launch_begin(p, "lsq_cta", s);
    k_lsq_cta<<<sms, CTA_THREADS, s5, s>>>(p->xs, p->phase, p->col_start, p->col_count, p->col_off, N, Ms, kp, mu,
                                           p->w64, p->w32, p->J, p->wide, p->big_list, p->counters);
    launch_end(p, s);
    return cudaGetLastError();
}

namespace {
HugeProblem huge_problem(const Plan* p) {
    HugeProblem h;
    h.xs = p->xs; h.ph = p->phase; h.col_start = p->col_start; h.col_count = p->col_count; h.col_off = p->col_off;
    h.w64 = p->w64; h.w32 = p->w32; h.J = p->J; h.wide = p->wide; h.counters = p->counters;
    h.big_list = p->big_list;
    h.N = (int)p->N; h.Ms = (int)p->Ms;
    h.kp = make_kernel_params(p);
    h.mu = p->tau * h.kp.diag;
    return h;
}
}  // namespace

size_t huge_problem_bytes() { return sizeof(HugeProblem); }

void huge_problems_fill(Plan* const* plans, int P, void* host) {
    HugeProblem* h = (HugeProblem*)host;
    for (int i = 0; i < P; ++i) h[i] = huge_problem(plans[i]);
}

// the triangles of every part's slots (HUGE_PART_MINB[k] per SM, of the part's largest column)
size_t huge_scratch_doubles(int slots, int nmax) {
    size_t tot = 0;
    for (int k = 0; k < HUGE_PARTS; ++k) {
        const size_t c = (size_t)std::min(nmax, HUGE_PART_LIMIT[k]);
        tot += (size_t)HUGE_PART_MINB[k] * slots * (c * (c + 1) / 2);
    }
    return tot;
}

cudaError_t run_precompute_huge(const void* probs, int P, int32_t* job_off, int32_t* order, int32_t* work,
                                double* scratch, int slots, int nmax, cudaStream_t s) {
    auto k0 = k_lsq_huge<HUGE_PART_LIMIT[0], HUGE_PART_THREADS[0], HUGE_PART_MINB[0]>;
    auto k1 = k_lsq_huge<HUGE_PART_LIMIT[1], HUGE_PART_THREADS[1], HUGE_PART_MINB[1]>;
    auto k2 = k_lsq_huge<HUGE_PART_LIMIT[2], HUGE_PART_THREADS[2], HUGE_PART_MINB[2]>;
    auto k3 = k_lsq_huge<HUGE_PART_LIMIT[3], HUGE_PART_THREADS[3], HUGE_PART_MINB[3]>;
    auto smem_of = [](int pmax) {
        return (size_t)(pmax * HUGE_PS + 2 * pmax) * sizeof(double) + (size_t)pmax * sizeof(double2);
    };
    cudaError_t e = set_smem(k0, smem_of(HUGE_PART_LIMIT[0]));
    if (e == cudaSuccess) e = set_smem(k1, smem_of(HUGE_PART_LIMIT[1]));
    if (e == cudaSuccess) e = set_smem(k2, smem_of(HUGE_PART_LIMIT[2]));
    if (e == cudaSuccess) e = set_smem(k3, smem_of(HUGE_PART_LIMIT[3]));
    if (e != cudaSuccess) return e;
    const HugeProblem* hp = (const HugeProblem*)probs;
    int32_t* hist = work;                  // nmax + 1 buckets (then their offsets, then cursors)
    int32_t* ticket = work + nmax + 1;     // the parts' tickets, then the splits
    int32_t* split = work + nmax + 1 + HUGE_PARTS;
    if ((e = cudaMemsetAsync(work, 0, (size_t)(nmax + 2 * HUGE_PARTS) * sizeof(int32_t), s)) != cudaSuccess)
        return e;
    k_huge_prefix<<<1, 1024, 0, s>>>(hp, P, job_off);
    k_job_hist<<<4 * slots, 256, 0, s>>>(hp, P, job_off, nmax, hist);
    k_job_scan<<<1, 1024, 0, s>>>(hist, nmax + 1);
    k_job_scatter<<<4 * slots, 256, 0, s>>>(hp, P, job_off, nmax, hist, order);
    k_job_split<<<1, 1, 0, s>>>(hist, nmax, split);
    int launches = 5;
    double* base = scratch;
    for (int k = 0; k < HUGE_PARTS; ++k) {
        const int lim = HUGE_PART_LIMIT[k];
        const size_t c = (size_t)std::min(nmax, lim);
        const size_t slot = c * (c + 1) / 2;
        const int ctas = HUGE_PART_MINB[k] * slots;
        if (k == HUGE_PARTS - 1 || nmax > HUGE_PART_LIMIT[k + 1]) {   // a part above nmax has no jobs
            if (k == 0) k0<<<ctas, HUGE_PART_THREADS[0], smem_of(lim), s>>>(hp, P, job_off, order, ticket, split, 0, base, slot, nmax);
            if (k == 1) k1<<<ctas, HUGE_PART_THREADS[1], smem_of(lim), s>>>(hp, P, job_off, order, ticket + 1, split, 1, base, slot, nmax);
            if (k == 2) k2<<<ctas, HUGE_PART_THREADS[2], smem_of(lim), s>>>(hp, P, job_off, order, ticket + 2, split, 2, base, slot, nmax);
            if (k == 3) k3<<<ctas, HUGE_PART_THREADS[3], smem_of(lim), s>>>(hp, P, job_off, order, ticket + 3, split, 3, base, slot, nmax);
            ++launches;
        }
        base += (size_t)ctas * slot;
    }
    count_launches(launches);
    return cudaGetLastError();
}

// ---- every problem of a batch in one launch per solver tier ----------------------------

namespace {

// The precompute counters of every problem (as run_precompute clears them for one).
__global__ void k_batch_clear_counters(const TierArgs* __restrict__ probs, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    int32_t* c = probs[p].counters;
    c[CNT_FALLBACK] = 0;
    c[CNT_UNSUPPORTED] = 0;
    c[CNT_LIST_A] = 0;
    c[CNT_BIG_LIST] = 0;
    c[CNT_TILES_MID] = 0;
    c[CNT_TILES_BIG] = 0;
    c[CNT_TILES_48] = 0;
    c[CNT_TILES_64] = 0;
    c[CNT_HUGE_LIST] = 0;
}

// off[p] = sum_{q < p} probs[q].counters[idx], off[P] = the total (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024)
k_batch_count_prefix(const TierArgs* __restrict__ probs, int P, int idx, int32_t* __restrict__ off) {
    __shared__ int32_t part[1024];
    const int per = (P + 1023) / 1024;
    const int a = min((int)threadIdx.x * per, P), b = min(a + per, P);
    int32_t sum = 0;
    for (int i = a; i < b; ++i) sum += probs[i].counters[idx];
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
        run += probs[i].counters[idx];
    }
    if (threadIdx.x == 1023) off[P] = part[1023];
}

}  // namespace

static TierArgs tier_args(const Plan* p) {
    TierArgs a;
    a.xs = p->xs; a.ph = p->phase; a.col_start = p->col_start; a.col_count = p->col_count; a.col_off = p->col_off;
    a.N = (int)p->N; a.Ms = (int)p->Ms;
    a.kp = make_kernel_params(p);
    a.mu0 = p->tau * a.kp.diag;
    a.w64 = p->w64; a.w32 = p->w32; a.J = p->J; a.wide = p->wide;
    a.tiles_mid = p->tiles_mid; a.tiles_big = p->tiles_big; a.tiles_48 = p->tiles_48; a.tiles_64 = p->tiles_64;
    a.list_a = p->list_a; a.big_list = p->big_list;
    a.counters = p->counters;
    return a;
}

size_t tier_args_bytes() { return sizeof(TierArgs); }

void tier_args_fill(Plan* const* plans, int P, void* host) {
    TierArgs* h = (TierArgs*)host;
    for (int i = 0; i < P; ++i) h[i] = tier_args(plans[i]);
}

cudaError_t run_precompute_batch(const void* probs_v, int P, const int32_t* tile_off, int total_tiles,
                                 int32_t* off_work, int sms, cudaStream_t s) {
    const TierArgs* probs = (const TierArgs*)probs_v;
    constexpr int A1 = LSQ_THREAD_NMAX1, A2 = LSQ_THREAD_NMAX2, A3 = LSQ_THREAD_NMAX3;
    constexpr int W1 = 5, G2 = LSQ_GROUP_G2, G3 = LSQ_GROUP_G3, W4 = 4;
    auto t1 = k_lsq_thread<A1, W1, true>;
    auto t2 = k_lsq_group<A2, G2, true>;
    auto t3 = k_lsq_group<A3, G3, true>;
    auto t4 = k_lsq_group<LSQ_GROUP_NMAX4, LSQ_GROUP_G4, true, LSQ_GROUP_TC4>;
    auto t5 = k_lsq_group<LSQ_WARP2_NMAX, LSQ_GROUP_G5, true, LSQ_GROUP_TC5>;
    auto k4 = k_lsq_warp<LSQ_WARP2_NMAX, W4, true>;
    const size_t s1 = W1 * tile_warp_bytes<A1>(), s2 = group_smem_bytes<A2>(), s3 = group_smem_bytes<A3>();
    const size_t st4 = group_smem_bytes<LSQ_GROUP_NMAX4, LSQ_GROUP_TC4>();
    const size_t st5 = group_smem_bytes<LSQ_WARP2_NMAX, LSQ_GROUP_TC5>();
    const size_t s4 = warp_smem_bytes<LSQ_WARP2_NMAX, W4>();
    cudaError_t e;
    if ((e = set_smem(t1, s1)) != cudaSuccess) return e;
    if ((e = set_smem(t2, s2)) != cudaSuccess) return e;
    if ((e = set_smem(t3, s3)) != cudaSuccess) return e;
    if ((e = set_smem(t4, st4)) != cudaSuccess) return e;
    if ((e = set_smem(t5, st5)) != cudaSuccess) return e;
    if ((e = set_smem(k4, s4)) != cudaSuccess) return e;
    int occ2 = 1, occ3 = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, t2, G2 * 32, s2)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ3, t3, G3 * 32, s3)) != cudaSuccess) return e;
    occ2 = std::max(occ2, 1);
    occ3 = std::max(occ3, 1);
    int32_t* off_mid = off_work;
    int32_t* off_big = off_work + (P + 1);
    int32_t* off_a = off_work + 2 * (P + 1);
    int32_t* off_48 = off_work + 3 * (P + 1);
    int32_t* off_64 = off_work + 4 * (P + 1);
    const KernelParams kp0 = {};
    k_batch_clear_counters<<<(P + 255) / 256, 256, 0, s>>>(probs, P);
    // routing tier: every tile of every problem, one warp each
    t1<<<(total_tiles + W1 - 1) / W1, W1 * 32, s1, s>>>(nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, kp0, 0.0,
                                                         nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr,
                                                         nullptr, nullptr, nullptr, nullptr, nullptr,
                                                         TierBatch{probs, tile_off, P});
    // group tiers and warp tier: the problems' routed lists, numbered by device prefixes
    k_batch_count_prefix<<<1, 1024, 0, s>>>(probs, P, CNT_TILES_MID, off_mid);
    t2<<<occ2 * sms, G2 * 32, s2, s>>>(nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, kp0, 0.0, nullptr, nullptr,
                                       nullptr, nullptr, nullptr, CNT_TILES_MID, nullptr, TierBatch{probs, off_mid, P});
    k_batch_count_prefix<<<1, 1024, 0, s>>>(probs, P, CNT_TILES_BIG, off_big);
    t3<<<occ3 * sms, G3 * 32, s3, s>>>(nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, kp0, 0.0, nullptr, nullptr,
                                       nullptr, nullptr, nullptr, CNT_TILES_BIG, nullptr, TierBatch{probs, off_big, P});
    k_batch_count_prefix<<<1, 1024, 0, s>>>(probs, P, CNT_TILES_48, off_48);
    t4<<<sms, LSQ_GROUP_TC4 * LSQ_GROUP_G4, st4, s>>>(nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, kp0, 0.0,
                                                      nullptr, nullptr, nullptr, nullptr, nullptr, CNT_TILES_48, nullptr,
                                                      TierBatch{probs, off_48, P});
    k_batch_count_prefix<<<1, 1024, 0, s>>>(probs, P, CNT_TILES_64, off_64);
    t5<<<sms, LSQ_GROUP_TC5 * LSQ_GROUP_G5, st5, s>>>(nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, kp0, 0.0,
                                                      nullptr, nullptr, nullptr, nullptr, nullptr, CNT_TILES_64, nullptr,
                                                      TierBatch{probs, off_64, P});
    k_batch_count_prefix<<<1, 1024, 0, s>>>(probs, P, CNT_LIST_A, off_a);
    k4<<<2 * sms, W4 * 32, s4, s>>>(nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, kp0, 0.0, nullptr, nullptr,
                                    nullptr, nullptr, nullptr, CNT_LIST_A, nullptr, CNT_BIG_LIST, nullptr,
                                    TierBatch{probs, off_a, P});
    count_launches(12);
    return cudaGetLastError();
}
