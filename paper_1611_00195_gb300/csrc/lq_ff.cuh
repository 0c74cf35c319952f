// Float-float numbers: an unevaluated sum hi + lo of two FP32 values with |lo| <= ulp(hi) / 2,
// about 48 significant bits, computed on the FP32 units.  On this GPU FP64 runs at 1/64 of the
// FP32 rate, so a float-float operation (a few to twenty FP32 instructions) is cheaper than the
// FP64 one it replaces while keeping rounding errors near 2^-47 instead of 2^-24.
//
//  * sum: Knuth's TwoSum of the high parts and of the low parts, each followed by Dekker's
//    renormalisation (the "accurate" double-word addition; Dekker, Numer. Math. 18 (1971) 224;
//    Joldes, Muller & Popescu, ACM TOMS 44 (2017), Algorithm 6), relative error below 3 u^2;
//  * product: the exact error of hi * hi from one FMA, the cross terms added to it, then the
//    renormalisation (Joldes, Muller & Popescu, Algorithm 11 without the lo * lo term), relative
//    error below 5 u^2;
//  * u = 2^-24.
// The compiler must not reassociate these FP32 operations: nvcc does not (no fast-math flags are
// used for this library), and no expression here has a product next to a sum that FMA
// contraction could fuse differently from the written order.
#pragma once
#include <cuda_runtime.h>

namespace lq {

// the FP32 / FP64 fma of the math library stays visible next to the float-float one below
using ::fma;

struct ff {
    float hi, lo;
    ff() = default;
    __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr ff(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ constexpr ff(float v) : hi(v), lo(0.f) {}
    // nearest FP32 and the FP32 nearest to the remainder (exact for |v| in the normal range
    // whenever v has at most 48 significant bits)
    __host__ __device__ ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return ff(s, e);
}
// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker)
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
    const float s = a + b;
    return ff(s, b - (s - a));
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }

__device__ __forceinline__ ff operator+(ff a, ff b) {
    ff s = ff_two_sum(a.hi, b.hi);
    const ff t = ff_two_sum(a.lo, b.lo);
    s = ff_fast_two_sum(s.hi, s.lo + t.hi);
    return ff_fast_two_sum(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

__device__ __forceinline__ ff operator*(ff a, ff b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);   // exact error of the rounded product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}

// a * b + c with the rounding of the product and of the sum (no single-rounding fused form)
__device__ __forceinline__ ff fma(ff a, ff b, ff c) { return a * b + c; }

// complex float-float (the kernels' C type); storage chunk: float4 (x.hi, x.lo, y.hi, y.lo)
struct cff {
    ff x, y;
};

__device__ __forceinline__ cff cff_from_chunk(float4 v) {
    cff r;
    r.x = ff(v.x, v.y);
    r.y = ff(v.z, v.w);
    return r;
}
__device__ __forceinline__ float4 cff_to_chunk(cff a) { return make_float4(a.x.hi, a.x.lo, a.y.hi, a.y.lo); }

}  // namespace lq
