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

// ---- double-float arithmetic on the float32 pipes
// Renormalisation assumes |a| >= |b| (Dekker's Fast2Sum).
LM_DEV void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
LM_DEV df df_make(float hi) { return df{hi, 0.f}; }
LM_DEV df df_neg(df a) { return df{-a.hi, -a.lo}; }
// sum with both words added error-free (accurate under cancellation)
LM_DEV df df_add(df a, df b) {
    float s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e = __fadd_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    df r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}
LM_DEV df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
LM_DEV df df_mul(df a, df b) {
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    df r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}
LM_DEV df df_mul_f(df a, float b) {
    float p, e;
    two_prod(a.hi, b, p, e);
    e = __fmaf_rn(a.lo, b, e);
    df r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}
// a - b*c, the update of elimination loops
LM_DEV df df_fms(df a, df b, df c) { return df_sub(a, df_mul(b, c)); }
// quotient by long division: two float32 quotient digits and a correction
LM_DEV df df_div(df a, df b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    df r = df_sub(a, df_mul_f(b, q1));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    r = df_sub(r, df_mul_f(b, q2));
    const float q3 = __fdiv_rn(r.hi, b.hi);
    df q;
    fast_two_sum(q1, q2, q.hi, q.lo);
    return df_add(q, df_make(q3));
}
// 1/sqrt(a) for a > 0: float32 seed, two Newton steps r <- r + r (1 - a r^2) / 2
LM_DEV df df_rsqrt(df a) {
    df r = df_make(rsqrtf(a.hi));
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const df e = df_sub(df_make(1.f), df_mul(a, df_mul(r, r)));
        r = df_add(r, df_mul_f(df_mul(r, e), 0.5f));
    }
    return r;
}
LM_DEV double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
LM_DEV bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

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
