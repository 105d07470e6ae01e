// teuk_df.cuh -- double-float numbers for the FP64-equivalent precision: a value hi + lo
// held in two FP32 numbers, |lo| <= ulp(hi)/2, about 48 significant bits (Dekker 1971),
// computed on the FP32 units with error-free transformations: Knuth's two-sum and the
// FMA-based exact product.  Every operation is written with explicit round-to-nearest
// intrinsics, so the compiler neither contracts nor reassociates them.
#pragma once
#include <cuda_runtime.h>

namespace teuk {

struct DF {
    float hi, lo;
    DF() = default;
    __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
    // nearest double-float of a double (exact for every double whose significand fits)
    __host__ __device__ constexpr DF(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ constexpr DF(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ constexpr double to_double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF operator-(DF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ DF operator+(DF x, DF y) {
    const DF s = df_two_sum(x.hi, y.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DF operator-(DF x, DF y) { return x + (-y); }
// product: the exact product of the high parts plus the cross terms
__device__ __forceinline__ DF operator*(DF x, DF y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return df_fast_two_sum(p, e);
}
// a * b + c with one normalisation: the product's error term joins c's low part
__device__ __forceinline__ DF tfma(DF a, DF b, DF c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const DF s = df_two_sum(p, c.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}
// x / 2 (exact)
__device__ __forceinline__ DF df_half(DF x) { return {0.5f * x.hi, 0.5f * x.lo}; }

}  // namespace teuk
