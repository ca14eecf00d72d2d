// Double-float ("df") arithmetic: a value is an unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, giving about 48 significand bits.
//
// GB300 executes FP64 FMAs at 1/64 of the FP32 rate with a 64-cycle
// dependent latency (measured on this part), so every quantity the method
// keeps beyond FP32 (transition-matrix powers, cross-tile state composition)
// is carried in df on the FP32 pipe instead.  The building blocks are the
// error-free transformations of Knuth (TwoSum), Dekker (Fast2Sum) and the
// FMA-based TwoProduct (see Muller et al., Handbook of Floating-Point
// Arithmetic, ch. 4 and 14); nvcc does not reassociate FP32 additions, so the
// sequences stay exact.
#pragma once

#include <cuda_runtime.h>

namespace sosf {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return df{s, e};
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    const float s = a + b;
    return df{s, b - (s - a)};
}

__device__ __forceinline__ df df_from(float a) { return df{a, 0.0f}; }

__device__ __forceinline__ df df_add(df a, df b) {
    df s = df_two_sum(a.hi, b.hi);
    const df t = df_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = df_fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return df_fast_two_sum(s.hi, s.lo);
}

// Cheaper addition (one TwoSum instead of two): the low parts are added
// without compensation, so the result carries about 2^-44 relative error
// unless the operands nearly cancel.  Used where terms of similar magnitude
// are summed (look-back compositions).
__device__ __forceinline__ df df_add_fast(df a, df b) {
    const df s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

// 2x2 matrix in df, row-major
struct dfm2 {
    df a, b, c, d;
};

__device__ __forceinline__ dfm2 dfm_mul(const dfm2& x, const dfm2& y) {
    return dfm2{df_add(df_mul(x.a, y.a), df_mul(x.b, y.c)), df_add(df_mul(x.a, y.b), df_mul(x.b, y.d)),
                df_add(df_mul(x.c, y.a), df_mul(x.d, y.c)), df_add(df_mul(x.c, y.b), df_mul(x.d, y.d))};
}

// The same product with the cheaper additions (about 2^-44 relative error per
// entry): for tables that are rounded to FP32 in the end.
__device__ __forceinline__ dfm2 dfm_mul_fast(const dfm2& x, const dfm2& y) {
    return dfm2{df_add_fast(df_mul(x.a, y.a), df_mul(x.b, y.c)),
                df_add_fast(df_mul(x.a, y.b), df_mul(x.b, y.d)),
                df_add_fast(df_mul(x.c, y.a), df_mul(x.d, y.c)),
                df_add_fast(df_mul(x.c, y.b), df_mul(x.d, y.d))};
}

// a / b: the quotient of the leading parts, corrected once by the remainder
// a - q1 b (the double-double division of Bailey's DDFUN/QD libraries,
// reduced to one correction step; about 2^-44 relative error).
__device__ __forceinline__ df df_div(df a, df b) {
    const float q1 = a.hi / b.hi;
    const df r = df_add(a, df_neg(df_mul(df{q1, 0.f}, b)));
    const float q2 = r.hi / b.hi;
    return df_fast_two_sum(q1, q2);
}

__device__ __forceinline__ dfm2 dfm_identity() {
    return dfm2{df{1.f, 0.f}, df{0.f, 0.f}, df{0.f, 0.f}, df{1.f, 0.f}};
}

// y = M u + c
__device__ __forceinline__ void dfm_affine(const dfm2& M, df u1, df u2, df c1, df c2, df& y1,
                                           df& y2) {
    y1 = df_add(df_add(df_mul(M.a, u1), df_mul(M.b, u2)), c1);
    y2 = df_add(df_add(df_mul(M.c, u1), df_mul(M.d, u2)), c2);
}

// y = M u + c with the cheaper additions
__device__ __forceinline__ void dfm_affine_fast(const dfm2& M, df u1, df u2, df c1, df c2, df& y1,
                                                df& y2) {
    y1 = df_add_fast(df_add_fast(df_mul(M.a, u1), df_mul(M.b, u2)), c1);
    y2 = df_add_fast(df_add_fast(df_mul(M.c, u1), df_mul(M.d, u2)), c2);
}

__device__ __forceinline__ float df_to_float(df a) { return a.hi + a.lo; }

// ---------------------------------------------------------------------------
// Double-float signal arithmetic for the sample recursions of channels run in
// extended precision.  A sample is (hi, lo); products use the FMA-based
// TwoProduct, sums of the leading parts Knuth's TwoSum, and every low-order
// term (the products' errors, the sums' errors, the cross terms hi*lo) is
// collected in one FP32 accumulator, then renormalised once (Fast2Sum).  The
// error of one such step is about 2^-44 of its operands.

// a0*x0 + a1*x1 + a2*x2 (coefficients and samples double-float)
__device__ __forceinline__ df df_dot3(df a0, df x0, df a1, df x1, df a2, df x2) {
    const float p0 = a0.hi * x0.hi, p1 = a1.hi * x1.hi, p2 = a2.hi * x2.hi;
    float c = fmaf(a0.hi, x0.hi, -p0);
    c += fmaf(a1.hi, x1.hi, -p1);
    c += fmaf(a2.hi, x2.hi, -p2);
    const df s1 = df_two_sum(p0, p1);
    const df s2 = df_two_sum(s1.hi, p2);
    c += s1.lo + s2.lo;
    c = fmaf(a0.hi, x0.lo, fmaf(a0.lo, x0.hi, c));
    c = fmaf(a1.hi, x1.lo, fmaf(a1.lo, x1.hi, c));
    c = fmaf(a2.hi, x2.lo, fmaf(a2.lo, x2.hi, c));
    return df_fast_two_sum(s2.hi, c);
}

// u - a1*y1 - a2*y2: one step of the all-pole recursion.  In a run, y1 is
// the previous step's result, so it enters last: the older term a2*y2 and
// every low-order term of a1*y1 are summed first, and only the TwoSum with
// a1*y1's rounded product and the final renormalisation follow y1.hi.
__device__ __forceinline__ df df_rec(df u, df a1, df y1, df a2, df y2) {
    const float p2 = a2.hi * y2.hi;
    const df s1 = df_two_sum(u.hi, -p2);
    float c = u.lo - fmaf(a2.hi, y2.hi, -p2);
    c = fmaf(-a2.hi, y2.lo, fmaf(-a2.lo, y2.hi, c));
    c += s1.lo;
    const float p1 = a1.hi * y1.hi;
    const float c1 = fmaf(-a1.hi, y1.lo, fmaf(-a1.lo, y1.hi, -fmaf(a1.hi, y1.hi, -p1)));
    const df s2 = df_two_sum(s1.hi, -p1);
    return df_fast_two_sum(s2.hi, (c + c1) + s2.lo);
}

// u - a1*y1 (the second sample of a run, one history term)
__device__ __forceinline__ df df_rec1(df u, df a1, df y1) {
    const float p1 = a1.hi * y1.hi;
    float c = u.lo - fmaf(a1.hi, y1.hi, -p1);
    const df s1 = df_two_sum(u.hi, -p1);
    c += s1.lo;
    c = fmaf(-a1.hi, y1.lo, fmaf(-a1.lo, y1.hi, c));
    return df_fast_two_sum(s1.hi, c);
}

}  // namespace sosf
