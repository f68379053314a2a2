// smol_dd.cuh - double-float arithmetic: a value is an unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= ulp(hi) / 2), about 48 significant bits, computed on the FP32
// pipes. GB300 executes FP32 at 64 times its FP64 rate, so the right-hand side of the
// FP64-accurate form (SMOL_DF64) runs its transforms, products and element-wise terms
// in this type and keeps only the state, its update, the error norm and the control in
// FP64.
//
// Built on the error-free transformations of Knuth (TAOCP vol. 2, Sec. 4.2.2: the sum
// of two floats as s + e exactly) and Dekker (1971: the product as p + e exactly, here
// with a fused multiply-add). Addition is the "sloppy" form (one two-sum on the high
// parts, the low parts added, one renormalisation): its error is below about
// 2^-46 (|a| + |b|), which bounds an FFT's error normwise as an FP64 rounding would,
// with a unit about 2^-46 instead of 2^-53. The exponent range is FP32's: callers scale
// their inputs (the per-transform power-of-two scaling of the FP32 form).
#pragma once
#include <cuda_runtime.h>

namespace smol {

struct dd {
    float hi, lo;
    dd() = default;
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dd(float x) : hi(x), lo(0.f) {}
    __host__ __device__ constexpr dd(int x) : hi((float)x), lo(0.f) {}  // exact for |x| < 2^24
    // The nearest double-float of an FP64 value (the high part rounded to FP32, the
    // remainder rounded again).
    __host__ __device__ dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ dd two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return dd(s, e);
}
// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker).
__device__ __forceinline__ dd fast_two_sum(float a, float b) {
    const float s = a + b;
    const float e = b - (s - a);
    return dd(s, e);
}

__device__ __forceinline__ dd operator+(dd a, dd b) {
    const dd s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
// p + e: the exact product of the high parts (fused multiply-add for the error), plus
// the cross terms; lo * lo is below the result's precision.
__device__ __forceinline__ dd operator*(dd a, dd b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ dd& operator+=(dd& a, dd b) {
    a = a + b;
    return a;
}

__device__ __forceinline__ dd shfl_down(dd v, int o) {
    return dd(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ float shfl_down(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }

// A pair of consecutive double-float values (16 bytes) and its loads.
struct __align__(16) dd2 {
    dd x, y;
};
__device__ __forceinline__ dd2 as_dd2(float4 v) {
    dd2 r;
    r.x = dd(v.x, v.y);
    r.y = dd(v.z, v.w);
    return r;
}

}  // namespace smol
