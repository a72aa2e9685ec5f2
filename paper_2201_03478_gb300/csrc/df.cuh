// df.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo
// of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.  On this
// GPU the FP32 pipes run 64 times faster than the FP64 pipe, so FP64-class
// accuracy is cheaper in pairs of floats for the long FMA chains of the two
// hot loops.
//
// The error-free transformations follow Dekker (1971) and Knuth (TAOCP vol. 2,
// 4.2.2): two_sum gives s + e = a + b exactly; fast_two_sum does the same
// when |a| >= |b|; two_prod gives p + e = a b exactly with one FMA.  Every
// step uses the _rn intrinsics so that the compiler neither contracts nor
// reassociates them.  Range: float exponents (values below ~1e-38 lose their
// low part), which the contraction's rescaled recurrence and the cube values
// stay well inside.
#pragma once

#include <cuda_runtime.h>

namespace sl {

struct __align__(8) dfl {
    float h, l;
};

__device__ __forceinline__ dfl df_make(float h, float l) { return dfl{h, l}; }

// double -> double-float (two roundings; exact to ~2^-48 relative)
__device__ __forceinline__ dfl df_from_d(double x) {
    const float h = __double2float_rn(x);
    return dfl{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to_d(dfl a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    dfl r;
    fast_two_sum(s, e, r.h, r.l);
    return r;
}
__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.h, -a.l}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    dfl r;
    fast_two_sum(p, e, r.h, r.l);
    return r;
}

// a b + c with one normalisation: the product's high part and c's high part
// meet in two_sum, every term of order 2^-24 relative goes to the low part.
__device__ __forceinline__ dfl df_fma(dfl a, dfl b, dfl c) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    float s, e2;
    two_sum(p, c.h, s, e2);
    e = __fadd_rn(e, __fadd_rn(e2, c.l));
    dfl r;
    fast_two_sum(s, e, r.h, r.l);
    return r;
}

// Accumulator for long sums of products: the high parts are summed with
// two_sum (exact), everything of order 2^-24 relative goes to lo; normalise
// once at the end (df_acc_get).
struct dacc {
    float h, l;
};
__device__ __forceinline__ void dacc_zero(dacc &s) { s.h = 0.f; s.l = 0.f; }
// s += a b
__device__ __forceinline__ void dacc_mac(dacc &s, dfl a, dfl b) {
    const float p = __fmul_rn(a.h, b.h);
    float pe = __fmaf_rn(a.h, b.h, -p);
    pe = __fmaf_rn(a.h, b.l, pe);
    pe = __fmaf_rn(a.l, b.h, pe);
    float t, e;
    two_sum(s.h, p, t, e);
    s.h = t;
    s.l = __fadd_rn(s.l, __fadd_rn(e, pe));
}
// s += a (a double-float)
__device__ __forceinline__ void dacc_add(dacc &s, dfl a) {
    float t, e;
    two_sum(s.h, a.h, t, e);
    s.h = t;
    s.l = __fadd_rn(s.l, __fadd_rn(e, a.l));
}
__device__ __forceinline__ dfl dacc_get(const dacc &s) {
    dfl r;
    fast_two_sum(s.h, s.l, r.h, r.l);
    return r;
}

}  // namespace sl
