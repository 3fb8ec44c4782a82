// Float-float sums on the fp32 pipe for the spreading and interpolation of "wide" columns
// (||b_l||_1 above WIDE_COLUMN_L1, whose terms cancel): the weight b = hi + lo is held as
// two fp32 values (lo = fp32(b - hi), formed in the precompute), each product is split
// exactly by an FMA, and the sum is carried as an unevaluated pair through Knuth's two-sum,
// about 44 significant bits without fp64 arithmetic.
#pragma once
#include "common.cuh"

// s + e = a + b exactly (the _rn intrinsics keep the compiler from reassociating or contracting)
INFFT_D void ff_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// sum_i (hi_i + lo_i) v_i for complex v
struct FFSum {
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    INFFT_D void add(float wh, float wl, float2 v) {
        const float tr = __fmul_rn(wh, v.x), ti = __fmul_rn(wh, v.y);
        const float lr = fmaf(wl, v.x, fmaf(wh, v.x, -tr)), li = fmaf(wl, v.y, fmaf(wh, v.y, -ti));
        float t, err;
        ff_two_sum(sr, tr, t, err);
        sr = t;
        cr += err + lr;
        ff_two_sum(si, ti, t, err);
        si = t;
        ci += err + li;
    }
    INFFT_D float2 value() const { return make_float2(sr + cr, si + ci); }
};
