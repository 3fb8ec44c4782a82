// Device helpers shared by the least-squares kernels of both optimisation
// problems (Sec. 3.2.1 and Sec. 3.2.2): the Dirichlet kernel kappa with the
// choice of Remark remark:Dirichlet_ansatz2 (eq:kernel_Dirichlet), node phases,
// the torus difference and the register Cholesky of the thread-per-column tier.
//
// Kernel values avoid library transcendentals on the common path: with per-node
// phases (sin, cos)(pi M x_j), sin(pi M (a - b)) follows by angle addition, and
// for |a - b| <= 1/32 the remaining factor cot(pi t) comes from the Taylor series
// of u cot u (coefficients 2^{2k} |B_{2k}| / (2k)!, B = Bernoulli numbers) and a
// Newton-Raphson reciprocal; pairs closer than a quarter period of sin(pi M t)
// use the Taylor series of sin(z)/z and cos(z) instead of the phases, so the
// cancellation in the angle addition never meets a tiny denominator.
#pragma once
#include <cmath>
#include <cstring>

#include "plan.h"

namespace {

struct KernelParams {
    double M;        // number of frequencies (as a double)
    double inv_Ms;   // 1 / M_sigma
    double diag;     // Re kappa(0)
    int sym;         // 0: full, 1: sym
    // near-pair evaluation of the full kernel (|t| <= 1/32), coefficients folded on the
    // host: Re kappa(t) = cx(t^2) * sin(pi M t) / t  with cx(t^2) = (u cot u) / (pi M_sigma),
    // u = pi t; and, for |M t| <= 1/4, Re kappa(t) = cx(t^2) * cs(t^2) with
    // cs(t^2) = pi M sin(z)/z, z = pi M t.
    double cx[7];
    double cs[9];
    int short_cot;   // 1: |pi t| of every near pair is so small that terms beyond cx[2] drop below 2^-56
    unsigned long long near_bits;   // bit pattern of 0.25 / M (|t| below it: sin(z)/z series)
    float* wlo;      // nnz_cap: low parts fp32(b - fp32(b)) of the float-float applies (or nullptr)
};

// Stores coefficient b of entry e in fp64, in fp32 and, when lo is given, the fp32 low part
// fp32(b - fp32(b)) that the fp32 applies use for wide columns (float-float).
INFFT_D void store_b(double* w64, float* w32, float* lo, int e, double b) {
    w64[e] = b;
    const float h = (float)b;
    w32[e] = h;
    if (lo) lo[e] = (float)(b - (double)h);
}

constexpr double PI = 3.141592653589793238462643383279502884;
constexpr double SMALL_T = 1.0 / 32.0;    // Taylor path for cot(pi t) below this |t|

// (sin, cos)(pi M z) with M z reduced modulo 2 exactly: M z = p + e with
// p = fl(M z) and e = fma(M, z, -p); p - 2 rint(p/2) is exact.
INFFT_D double2 phase_of(double M, double z) {
    const double p = M * z;
    const double e = fma(M, z, -p);
    const double r = p - 2.0 * rint(0.5 * p);
    double s, c;
    sincospi(r + e, &s, &c);
    return make_double2(s, c);
}

// 1/u to full fp64 precision: fp32 seed, two Newton-Raphson steps r <- r (2 - u r).
INFFT_D double recip(double u) {
    double r = (double)__frcp_rn((float)u);
    double e = fma(-u, r, 1.0);
    r = fma(r, e, r);
    e = fma(-u, r, 1.0);
    return fma(r, e, r);
}

// Torus difference a - b in [-1/2, 1/2]: shifting each operand by 1/2 before
// subtracting keeps the difference of two points close across the seam x = +-1/2
// exact (subtracting first and wrapping afterwards loses ~11 digits there and
// can make Re G_l + mu I indefinite).
INFFT_D double torus_diff(double a, double b) {
    double t = a - b;
    if (t > 0.5) t = (a - 0.5) - (b + 0.5);
    else if (t < -0.5) t = (a + 0.5) - (b - 0.5);
    return t;
}

// Re kappa(t) with library transcendentals (any t in [-1/2, 1/2]).
INFFT_D double re_kappa_general(double t, const KernelParams& kp) {
    double s, c;
    sincospi(t, &s, &c);
    if (kp.sym) return sinpi((kp.M - 1.0) * t) / s * kp.inv_Ms;
    return c * sinpi(kp.M * t) / s * kp.inv_Ms;
}

// Re kappa(a - b); pa, pb = (sin, cos)(pi M a), (sin, cos)(pi M b).
INFFT_D double re_kappa(double a, double b, double2 pa, double2 pb, const KernelParams& kp) {
    const double t = torus_diff(a, b);
    if (t == 0.0) return kp.diag;
    if (fabs(t) > SMALL_T) return re_kappa_general(t, kp);
    const double u = PI * t;
    const double w = u * u;
    // u cot u = 1 - w/3 - w^2/45 - 2w^3/945 - w^4/4725 - 2w^5/93555 - 1382 w^6/638512875
    double xc = fma(w, -1382.0 / 638512875.0, -2.0 / 93555.0);
    xc = fma(w, xc, -1.0 / 4725.0);
    xc = fma(w, xc, -2.0 / 945.0);
    xc = fma(w, xc, -1.0 / 45.0);
    xc = fma(w, xc, -1.0 / 3.0);
    xc = fma(w, xc, 1.0);
    const double y = kp.M * t;
    double s_over_u, cm = 0.0;
    if (fabs(y) <= 0.25) {
        // sin(pi M t)/(pi t) = M sin(z)/z and cos(z), z = pi M t, |z| <= pi/4
        const double z = PI * y;
        const double v = z * z;
        double sz = fma(v, 1.0 / 355687428096000.0, -1.0 / 1307674368000.0);
        sz = fma(v, sz, 1.0 / 6227020800.0);
        sz = fma(v, sz, -1.0 / 39916800.0);
        sz = fma(v, sz, 1.0 / 362880.0);
        sz = fma(v, sz, -1.0 / 5040.0);
        sz = fma(v, sz, 1.0 / 120.0);
        sz = fma(v, sz, -1.0 / 6.0);
        sz = fma(v, sz, 1.0);
        s_over_u = kp.M * sz;
        if (kp.sym) {
            double cz = fma(v, -1.0 / 6402373705728000.0, 1.0 / 20922789888000.0);
            cz = fma(v, cz, -1.0 / 87178291200.0);
            cz = fma(v, cz, 1.0 / 479001600.0);
            cz = fma(v, cz, -1.0 / 3628800.0);
            cz = fma(v, cz, 1.0 / 40320.0);
            cz = fma(v, cz, -1.0 / 720.0);
            cz = fma(v, cz, 1.0 / 24.0);
            cz = fma(v, cz, -0.5);
            cm = fma(v, cz, 1.0);
        }
    } else {
        // sin(pi M (a - b)) = sin A cos B - cos A sin B; M is even, so the torus wrap of
        // t changes neither sin(pi M t) nor cos(pi M t)
        const double sm = fma(pa.x, pb.y, -pa.y * pb.x);
        s_over_u = sm * recip(u);
        if (kp.sym) cm = fma(pa.y, pb.y, pa.x * pb.x);
    }
    double g = xc * s_over_u;        // cot(pi t) sin(pi M t)
    if (kp.sym) g -= cm;             // sin(pi (M-1) t) / sin(pi t)
    return g * kp.inv_Ms;
}

// (i, j), j <= i, of the e-th entry of a row-major lower triangle
INFFT_D void tri_index(int e, int& i, int& j) {
    int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    while (r * (r + 1) / 2 > e) --r;
    i = r;
    j = e - r * (r + 1) / 2;
}

INFFT_D int trow(int i) { return i * (i + 1) / 2; }   // packed lower-triangle row start

INFFT_D double col_t(int p, int Ms) { return (double)(p - Ms / 2) / (double)Ms; }   // l / M_sigma

// Re kappa(t) of the full kernel for a pair known to be near (|t| <= 1/32, t taken
// without a seam): u cot u and sin(z)/z by their Taylor series (coefficients folded
// on the host), sin(pi M t) by angle addition of the phases, branches decided on
// the bit pattern of |t| so that no fp64 comparison is issued.
INFFT_D double kappa_near(double t, double2 pa, double2 pb, const KernelParams& kp) {
    const unsigned long long tb = (unsigned long long)__double_as_longlong(t) & 0x7fffffffffffffffULL;
    if (tb == 0ULL) return kp.diag;
    const double t2 = t * t;
    double xc;
    if (kp.short_cot) {   // uniform across the launch
        xc = fma(t2, kp.cx[2], kp.cx[1]);
        xc = fma(t2, xc, kp.cx[0]);
    } else {
        xc = fma(t2, kp.cx[6], kp.cx[5]);
        xc = fma(t2, xc, kp.cx[4]);
        xc = fma(t2, xc, kp.cx[3]);
        xc = fma(t2, xc, kp.cx[2]);
        xc = fma(t2, xc, kp.cx[1]);
        xc = fma(t2, xc, kp.cx[0]);
    }
    if (tb <= kp.near_bits) {
        double sz = fma(t2, kp.cs[8], kp.cs[7]);
        sz = fma(t2, sz, kp.cs[6]);
        sz = fma(t2, sz, kp.cs[5]);
        sz = fma(t2, sz, kp.cs[4]);
        sz = fma(t2, sz, kp.cs[3]);
        sz = fma(t2, sz, kp.cs[2]);
        sz = fma(t2, sz, kp.cs[1]);
        sz = fma(t2, sz, kp.cs[0]);
        return xc * sz;
    }
    const double sm = fma(pa.x, pb.y, -pa.y * pb.x);    // sin(pi M (a - b))
    return xc * sm * recip(t);
}

// Up-looking Cholesky of the packed triangle T (stride 32) fused with the forward
// solve, then the backward solve, for n <= NMAX.  Fully unrolled: the current row
// of L, the reciprocal pivots and the right-hand side / solution (v: r, then y,
// then b, in place) stay in registers; the shared-memory traffic is loads of
// earlier rows (rows of L overwrite rows of T).  Returns false on a non-positive pivot.
template <int NMAX>
INFFT_D bool chol_solve(double* T, int n, double (&v)[NMAX], double& ysq) {
    double invd[NMAX];
    bool ok = true;
    ysq = 0.0;
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        if (i < n) {
            double li[NMAX];
#pragma unroll
            for (int j = 0; j < i; ++j) {
                double a0 = T[(trow(i) + j) * 32], a1 = 0.0;
#pragma unroll
                for (int k = 0; k < j; k += 2) {
                    a0 = fma(-li[k], T[(trow(j) + k) * 32], a0);
                    if (k + 1 < j) a1 = fma(-li[k + 1], T[(trow(j) + k + 1) * 32], a1);
                }
                li[j] = (j > 1 ? a0 + a1 : a0) * invd[j];
                T[(trow(i) + j) * 32] = li[j];
            }
            double d0 = T[(trow(i) + i) * 32], d1 = 0.0, y0 = v[i], y1 = 0.0;
#pragma unroll
            for (int k = 0; k < i; k += 2) {
                d0 = fma(-li[k], li[k], d0);
                y0 = fma(-li[k], v[k], y0);
                if (k + 1 < i) {
                    d1 = fma(-li[k + 1], li[k + 1], d1);
                    y1 = fma(-li[k + 1], v[k + 1], y1);
                }
            }
            const double d = i > 1 ? d0 + d1 : d0;
            ok = ok && (d > 0.0) && isfinite(d);
            invd[i] = rsqrt(d);
            T[(trow(i) + i) * 32] = invd[i];
            v[i] = (i > 1 ? y0 + y1 : y0) * invd[i];
            ysq = fma(v[i], v[i], ysq);
        }
    }
#pragma unroll
    for (int k = NMAX - 1; k >= 0; --k) {
        if (k < n) {
            double a0 = v[k], a1 = 0.0;
#pragma unroll
            for (int i = k + 1; i < NMAX; i += 2) {
                if (i < n) a0 = fma(-T[(trow(i) + k) * 32], v[i], a0);
                if (i + 1 < NMAX && i + 1 < n) a1 = fma(-T[(trow(i + 1) + k) * 32], v[i + 1], a1);
            }
            v[k] = (a0 + a1) * invd[k];
        }
    }
    return ok;
}

// One problem's buffers for the batch mode of the solver tiers (lsq.cu): one launch of a tier
// covers the work items of all problems of a batch.
struct TierArgs {
    const double* xs;
    const double2* ph;
    const int32_t* col_start;
    const int32_t* col_count;
    const int32_t* col_off;
    int N, Ms;
    KernelParams kp;
    double mu0;
    double* w64;
    float* w32;
    double* J;
    uint8_t* wide;
    int32_t* tiles_mid;
    int32_t* tiles_big;
    int32_t* tiles_48;
    int32_t* tiles_64;
    int32_t* list_a;
    int32_t* big_list;
    int32_t* counters;
};

// Batch mode of a tier launch: probs == nullptr for a single-problem launch; otherwise P
// problems whose work items are numbered by the prefix off (P + 1 entries on the device).
struct TierBatch {
    const TierArgs* probs;
    const int32_t* off;
    int P;
};

// The problem of global work item `it`: the largest p with off[p] <= it (off non-decreasing).
INFFT_D int batch_problem(const int32_t* __restrict__ off, int P, int it) {
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= it) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Kernel constants of a plan (host side).
// Device view of one plan for the large-column tier (lsq.cu).
struct HugeProblem {
    const double* xs;
    const double2* ph;
    const int32_t* col_start;
    const int32_t* col_count;
    const int32_t* col_off;
    double* w64;
    float* w32;
    double* J;
    uint8_t* wide;
    int32_t* counters;
    const int32_t* big_list;
    int N, Ms;
    double mu;
    KernelParams kp;
};

inline KernelParams make_kernel_params(const Plan* p) {
    const int64_t Ms = p->Ms;
    KernelParams kp;
    kp.wlo = p->wlo;
    kp.M = (double)p->M;
    kp.inv_Ms = 1.0 / (double)Ms;
    kp.sym = (p->kernel == INFFT_KERNEL_SYM);
    kp.diag = (kp.sym ? (double)(p->M - 1) : (double)p->M) / (double)Ms;
    {
        // u cot u = sum_k c_k u^{2k} (Bernoulli numbers); folded: cx_k = c_k pi^{2k} / (pi M_sigma)
        const double c[7] = {1.0, -1.0 / 3.0, -1.0 / 45.0, -2.0 / 945.0, -1.0 / 4725.0, -2.0 / 93555.0,
                             -1382.0 / 638512875.0};
        const double pi = 3.141592653589793238462643383279502884;
        double pw = 1.0;
        for (int k = 0; k < 7; ++k) {
            kp.cx[k] = c[k] * pw / (pi * (double)Ms);
            pw *= pi * pi;
        }
        // pi M sin(z)/z = pi M sum_k (-1)^k z^{2k} / (2k+1)!, z = pi M t
        const double a = pi * (double)p->M;
        double term = a, fact = 1.0;
        for (int k = 0; k < 9; ++k) {
            kp.cs[k] = term / fact;
            term *= -a * a;
            fact *= (double)(2 * k + 2) * (double)(2 * k + 3);
        }
        const double nb = 0.25 / (double)p->M;
        memcpy(&kp.near_bits, &nb, sizeof nb);
        // The thread and group tiers call kappa_near only for pairs inside a tile's
        // node union (32 consecutive columns: cells l0 - m .. l0 + 31 + m), so
        // |t| < (2m + 34)/M_sigma.  The first dropped term of u cot u is then
        // |c_3| u^6 with u = pi |t|; three terms suffice when it is below 2^-56.
        const double u = pi * (double)(2 * p->m + 34) / (double)Ms;
        const double w3 = u * u * u * u * u * u;
        kp.short_cot = (2.0 / 945.0) * w3 < std::ldexp(1.0, -56);
    }
    return kp;
}

}  // namespace
