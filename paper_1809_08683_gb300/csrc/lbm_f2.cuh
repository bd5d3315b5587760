// Packed pair of FP32 lanes for the paired-node fused kernel.
//
// Blackwell executes FP32 multiply, add and fused multiply-add on pairs of
// values in one instruction (__fmul2_rn, __fadd2_rn, __ffma2_rn).  `f2`
// carries the same quantity of two neighbouring lattice nodes; the node
// arithmetic of lbm_node.cuh is instantiated with R = f2 unchanged.  A
// product is kept pending (`f2p`) until it meets an addition, so that
// a * b + c becomes one packed FMA, as scalar contraction would make it.
// Every lane rounds exactly like the scalar FP32 operation it replaces.
#pragma once

#include <cuda_runtime.h>

#include "lbm_node.cuh"

namespace lbm {

struct f2p;

struct f2 {
    float2 v;
    __device__ __forceinline__ f2() {}
    __device__ __forceinline__ f2(float a) : v(make_float2(a, a)) {}
    __device__ __forceinline__ f2(double a) : v(make_float2((float)a, (float)a)) {}
    __device__ __forceinline__ f2(int a) : v(make_float2((float)a, (float)a)) {}
    __device__ __forceinline__ f2(float2 x) : v(x) {}
    __device__ __forceinline__ f2(const f2p& p);
};

struct f2p {  // pending product a * b
    float2 a, b;
};

__device__ __forceinline__ float2 neg2(float2 x) { return make_float2(-x.x, -x.y); }

__device__ __forceinline__ f2::f2(const f2p& p) : v(__fmul2_rn(p.a, p.b)) {}

__device__ __forceinline__ f2p operator*(const f2& a, const f2& b) { return f2p{a.v, b.v}; }
__device__ __forceinline__ f2p operator*(const f2p& p, const f2& c) { return f2p{__fmul2_rn(p.a, p.b), c.v}; }
__device__ __forceinline__ f2p operator*(const f2& c, const f2p& p) { return f2p{c.v, __fmul2_rn(p.a, p.b)}; }
__device__ __forceinline__ f2p operator*(const f2p& p, const f2p& q) {
    return f2p{__fmul2_rn(p.a, p.b), __fmul2_rn(q.a, q.b)};
}

__device__ __forceinline__ f2 operator+(const f2& a, const f2& b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator-(const f2& a, const f2& b) { return f2(__fadd2_rn(a.v, neg2(b.v))); }
__device__ __forceinline__ f2 operator-(const f2& a) { return f2(neg2(a.v)); }
__device__ __forceinline__ f2p operator-(const f2p& p) { return f2p{neg2(p.a), p.b}; }

__device__ __forceinline__ f2 operator+(const f2p& p, const f2& c) { return f2(__ffma2_rn(p.a, p.b, c.v)); }
__device__ __forceinline__ f2 operator+(const f2& c, const f2p& p) { return f2(__ffma2_rn(p.a, p.b, c.v)); }
__device__ __forceinline__ f2 operator-(const f2p& p, const f2& c) { return f2(__ffma2_rn(p.a, p.b, neg2(c.v))); }
__device__ __forceinline__ f2 operator-(const f2& c, const f2p& p) { return f2(__ffma2_rn(neg2(p.a), p.b, c.v)); }
__device__ __forceinline__ f2 operator+(const f2p& p, const f2p& q) {
    return f2(__ffma2_rn(p.a, p.b, __fmul2_rn(q.a, q.b)));
}
__device__ __forceinline__ f2 operator-(const f2p& p, const f2p& q) {
    return f2(__ffma2_rn(p.a, p.b, neg2(__fmul2_rn(q.a, q.b))));
}

__device__ __forceinline__ f2& operator+=(f2& a, const f2& b) { return a = a + b; }
__device__ __forceinline__ f2& operator-=(f2& a, const f2& b) { return a = a - b; }

// Per-lane operations without a packed form.
__device__ __forceinline__ f2 fdiv(const f2& a, const f2& b) {
    return f2(make_float2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y)));
}
__device__ __forceinline__ f2 sqrt(const f2& a) { return f2(make_float2(sqrtf(a.v.x), sqrtf(a.v.y))); }

__device__ __forceinline__ f2 cs_dev(const f2& b, const f2& rho0, const f2& Rg, const f2& rho_d, const f2& T,
                                     const f2& T_d) {
    return f2(make_float2((float)cs_dev1(b.v.x, rho0.v.x, Rg.v.x, rho_d.v.x, T.v.x, T_d.v.x),
                          (float)cs_dev1(b.v.y, rho0.v.y, Rg.v.y, rho_d.v.y, T.v.y, T_d.v.y)));
}

}  // namespace lbm
