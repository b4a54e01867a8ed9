// Shared device helpers of the LinMin CUDA path (sm_103a).
//
// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of
// two float32 words with |lo| <= ulp(hi)/2, which carries about 48 bits of
// significand.  The transformations below are the classic error-free ones:
//   two_sum  — Knuth's TwoSum: s + e == a + b exactly (6 flops, any order);
//   two_prod — with a fused multiply-add, p + e == a * b exactly (2 flops),
//              as in Ogita, Rump & Oishi, "Accurate sum and dot product"
//              (SIAM J. Sci. Comput. 26, 2005), algorithm TwoProduct with FMA.
// They are used where the fully constrained problem needs more than float32:
// the projection c = S W^2 y and the KKT residual G x - c near the solution
// (cancellation of O(1) terms down to O(1e-9) in the scaled problem).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define LM_DEV __device__ __forceinline__

namespace lm {

struct df { float hi, lo; };

LM_DEV void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float aa = __fsub_rn(s, bb);
    e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}

LM_DEV void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Accumulator for sum_k a_k * b_k in double-float: s holds the running
// float32 sum of the rounded products, c collects every rounding error
// (product errors and addition errors).  Final value ~ s + c (Dot2).
struct dot2 {
    float s = 0.f, c = 0.f;
    LM_DEV void add_prod(float a, float b) {
        float p, ep, t, es;
        two_prod(a, b, p, ep);
        two_sum(s, p, t, es);
        s = t;
        c = __fadd_rn(c, __fadd_rn(ep, es));
    }
    // add a small correction term whose own rounding is negligible
    LM_DEV void add_small(float v) { c = __fadd_rn(c, v); }
    LM_DEV void add_df(df v) {
        float t, es;
        two_sum(s, v.hi, t, es);
        s = t;
        c = __fadd_rn(c, __fadd_rn(v.lo, es));
    }
    LM_DEV df result() const {
        df r;
        two_sum(s, c, r.hi, r.lo);
        return r;
    }
};

// Split an fp64 value into hi + lo float32 words.
LM_DEV df split_double(double v) {
    df r;
    r.hi = __double2float_rn(v);
    r.lo = __double2float_rn(v - (double)r.hi);
    return r;
}

LM_DEV float group_sum(float v, int G) {
    for (int off = 1; off < G; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
LM_DEV float group_max(float v, int G) {
    for (int off = 1; off < G; off <<= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}
LM_DEV float group_min(float v, int G) {
    for (int off = 1; off < G; off <<= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

}  // namespace lm
