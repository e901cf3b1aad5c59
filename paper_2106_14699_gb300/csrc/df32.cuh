// Two-term FP32 ("double-float") numbers: value = hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits from FP32 units.  Used for the split-precision
// transforms, where FP32's 24 bits cannot keep every count's rounding residual
// under the guard but FP64 is slow on GB300.
//
// Addition follows Knuth's TwoSum (an exact error-free sum of two floats) and
// renormalises with Dekker's FastTwoSum; multiplication takes the exact product
// error from an FMA (p = a*b, e = fma(a, b, -p)).  These are the standard
// error-free transformations of floating-point arithmetic.
#pragma once
#include <cuda_runtime.h>

namespace cmif {

struct df32 {
    float hi, lo;
    __host__ __device__ constexpr df32() : hi(0.f), lo(0.f) {}
    __host__ __device__ constexpr df32(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr df32(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ constexpr df32(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ df32 df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ df32 df_fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df32 operator+(df32 x, df32 y) {
    df32 s = df_two_sum(x.hi, y.hi);
    const df32 t = df_two_sum(x.lo, y.lo);
    s = df_fast_two_sum(s.hi, s.lo + t.hi);
    return df_fast_two_sum(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ df32 operator-(df32 x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df32 operator-(df32 x, df32 y) { return x + (-y); }
__device__ __forceinline__ df32 operator*(df32 x, df32 y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df32 fabs(df32 x) { return x.hi < 0.f ? -x : x; }

}  // namespace cmif
