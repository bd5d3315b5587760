// Double-float ("float-float") arithmetic for the FP64-storage fused kernel.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, which carries about 48 significant bits.  On GB300
// the FP64 pipe runs at about 1/58 of the FP32 rate, and a double-float
// multiply-add costs about eleven FP32 instructions, so the per-node
// arithmetic of lbm_node.cuh, instantiated with R = ff64 unchanged, runs
// several times faster than in native FP64 while the DFs stay stored in
// FP64.  The algorithms are the error-free transformations of Knuth
// (two-sum), Dekker (fast two-sum) and the FMA-based exact product, combined
// as in the double-double literature (Hida, Li and Bailey): every operation
// is accurate to a few units in 2^-48 relative, except for subnormal
// magnitudes, which the lattice quantities never reach.
#pragma once

#include <cuda_runtime.h>

#include "lbm_node.cuh"

namespace lbm {

struct ff64 {
    float hi, lo;
    __host__ __device__ __forceinline__ ff64() {}
    __host__ __device__ __forceinline__ constexpr ff64(float h, float l) : hi(h), lo(l) {}
    // literal and parameter conversions; folded at compile time for constants
    __host__ __device__ __forceinline__ constexpr ff64(double a) : hi((float)a), lo((float)(a - (double)(float)a)) {}
    __host__ __device__ __forceinline__ constexpr ff64(float a) : hi(a), lo(0.0f) {}
    __host__ __device__ __forceinline__ constexpr ff64(int a) : hi((float)a), lo(0.0f) {}
    __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
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

__device__ __forceinline__ ff64& operator+=(ff64& a, const ff64& b) { return a = a + b; }
__device__ __forceinline__ ff64& operator-=(ff64& a, const ff64& b) { return a = a - b; }

// a / b: an FP32 quotient refined twice against the exact residual
__device__ __forceinline__ ff64 fdiv(const ff64& a, const ff64& b) {
    const float r = 1.0f / b.hi;
    const float q1 = a.hi * r;
    ff64 rem = a - b * ff64(q1, 0.0f);
    const float q2 = rem.hi * r;
    rem = rem - b * ff64(q2, 0.0f);
    const float q3 = rem.hi * r;
    return fast_two_sum(q1, q2) + ff64(q3, 0.0f);
}

// sqrt(a) for a > 0: the FP32 root refined by one Newton step in
// double-float (Karp and Markstein)
__device__ __forceinline__ ff64 sqrt(const ff64& a) {
    const float x = rsqrtf(a.hi);
    const float y = a.hi * x;
    const ff64 yy = ff64(y, 0.0f) * ff64(y, 0.0f);
    const float corr = (a - yy).hi * (x * 0.5f);
    return fast_two_sum(y, corr);
}

__device__ __forceinline__ bool isfinite(const ff64& a) { return ::isfinite(a.hi); }

__device__ __forceinline__ ff64 cs_dev(const ff64& b, const ff64& rho0, const ff64& Rg, const ff64& rho_d, const ff64& T,
                                       const ff64& T_d) {
    return ff64(cs_dev1((double)b, (double)rho0, (double)Rg, (double)rho_d, (double)T, (double)T_d));
}

}  // namespace lbm
