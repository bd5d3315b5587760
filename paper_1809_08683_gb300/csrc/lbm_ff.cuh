// Double-float ("float-float") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, which carries about
// 48 significant bits in FP32 instructions.  lbm_peak_rates measures its
// multiply-add rate next to the FP64 and FP32 FMA rates, the figures that
// decide whether FP64-accurate node arithmetic is cheaper in FP32 pairs than
// on GB300's FP64 pipe.  The algorithms are the error-free transformations
// of Knuth (two-sum), Dekker (fast two-sum) and the FMA-based exact
// product, combined as in the double-double literature (Hida, Li and
// Bailey): every operation is accurate to a few units in 2^-48 relative,
// except for subnormal magnitudes.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct ff64 {
    float hi, lo;
    __host__ __device__ __forceinline__ ff64() {}
    __host__ __device__ __forceinline__ constexpr ff64(float h, float l) : hi(h), lo(l) {}
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ ff64 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return ff64(s, e);
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ ff64 fast_two_sum(float a, float b) {
    const float s = a + b;
    return ff64(s, b - (s - a));
}

__device__ __forceinline__ ff64 operator+(const ff64& a, const ff64& b) {
    ff64 s = two_sum(a.hi, b.hi);
    const ff64 t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(s.hi, s.lo + t.lo);
}

__device__ __forceinline__ ff64 operator-(const ff64& a) { return ff64(-a.hi, -a.lo); }
__device__ __forceinline__ ff64 operator-(const ff64& a, const ff64& b) { return a + (-b); }

// product: hi * hi exactly through the FMA, the cross terms added in FP32
__device__ __forceinline__ ff64 operator*(const ff64& a, const ff64& b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

}  // namespace lbm
