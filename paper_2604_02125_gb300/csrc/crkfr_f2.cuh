// crkfr_f2.cuh -- packed FP32 pairs for the FP32 pair-flux form (sm_103a).
//
// f2 holds two independent FP32 values and maps + - * and fused multiply-add
// onto the packed FP32x2 instructions of this GPU (one instruction for both
// halves).  The volume kernel puts the pair flux of an x-line in one half and
// that of a y-line in the other, so the whole two-point flux code of the
// physics header, instantiated with R = f2, evaluates two fluxes per
// instruction stream.  A product followed by an addition is contracted into
// one fused multiply-add, as the compiler does for scalar code.
#pragma once
#include <cuda_runtime.h>

#include "crkfr_physics.cuh"

namespace crk {

struct f2 {
  float2 v;
  f2() = default;
  __device__ __forceinline__ f2(float2 x) : v(x) {}
  __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
  // broadcast of a constant (R(0.5), R(2) in the generic physics code)
  __device__ __forceinline__ f2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ f2(double a) : v(make_float2((float)a, (float)a)) {}
  __device__ __forceinline__ f2(int a) : v(make_float2((float)a, (float)a)) {}
};

// a product waiting for an addend: x * y + z becomes one FFMA2
struct f2prod {
  f2 a, b;
  __device__ __forceinline__ operator f2() const { return f2(__fmul2_rn(a.v, b.v)); }
};

__device__ __forceinline__ f2prod operator*(f2 a, f2 b) { return f2prod{a, b}; }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator-(f2 a) { return f2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return f2(__fadd2_rn(a.v, (-b).v)); }
__device__ __forceinline__ f2 operator+(f2prod p, f2 c) { return f2(__ffma2_rn(p.a.v, p.b.v, c.v)); }
__device__ __forceinline__ f2 operator+(f2 c, f2prod p) { return f2(__ffma2_rn(p.a.v, p.b.v, c.v)); }
__device__ __forceinline__ f2 operator-(f2prod p, f2 c) { return f2(__ffma2_rn(p.a.v, p.b.v, (-c).v)); }
__device__ __forceinline__ f2 operator-(f2 c, f2prod p) { return f2(__ffma2_rn((-p.a).v, p.b.v, c.v)); }
__device__ __forceinline__ f2 operator+(f2prod p, f2prod q) { return f2(__ffma2_rn(p.a.v, p.b.v, f2(q).v)); }
__device__ __forceinline__ f2 operator-(f2prod p, f2prod q) { return f2(__ffma2_rn(p.a.v, p.b.v, (-f2(q)).v)); }
__device__ __forceinline__ f2prod operator*(f2prod p, f2 b) { return f2prod{f2(p), b}; }
__device__ __forceinline__ f2prod operator*(f2 b, f2prod p) { return f2prod{b, f2(p)}; }
__device__ __forceinline__ f2prod operator*(f2prod p, f2prod q) { return f2prod{f2(p), f2(q)}; }
__device__ __forceinline__ f2& operator+=(f2& a, f2 b) { return a = a + b; }
__device__ __forceinline__ f2& operator+=(f2& a, f2prod p) { return a = p + a; }
__device__ __forceinline__ f2& operator-=(f2& a, f2 b) { return a = a - b; }
__device__ __forceinline__ f2& operator*=(f2& a, f2 b) { return a = f2(a * b); }

__device__ __forceinline__ f2 fast_rcp(f2 x) { return f2(fast_rcp(x.v.x), fast_rcp(x.v.y)); }

__device__ __forceinline__ f2 series_F(f2 u) {
  const f2 c9(1.0f / 9.0f), c7(1.0f / 7.0f), c5(1.0f / 5.0f), c3(1.0f / 3.0f), c1(1.0f);
  return u * (u * (u * (u * c9 + c7) + c5) + c3) + c1;
}

__device__ __forceinline__ f2 series_invF(f2 u) {
  const f2 c4(-428.0f / 14175.0f), c3(-44.0f / 945.0f), c2(-4.0f / 45.0f), c1(-1.0f / 3.0f), c0(1.0f);
  return u * (u * (u * (u * c4 + c3) + c2) + c1) + c0;
}

// L(a1,b1) and 1/L(a2,b2) in both halves, as the scalar FP32 version: one
// reciprocal per half, one branch for all four series tests (the common
// case), otherwise each half takes the scalar route.
__device__ __forceinline__ void logmean_pair(f2 a1, f2 b1, f2 a2, f2 b2, f2& L1, f2& iL2) {
  const f2 s1 = a1 + b1, d1 = a1 - b1, s2 = a2 + b2, d2 = a2 - b2;
  const f2 r = fast_rcp(f2(s1 * s2));
  const f2 rs1 = s2 * r, rs2 = s1 * r;
  const f2 q1 = d1 * rs1, q2 = d2 * rs2;
  const f2 u1 = q1 * q1, u2 = q2 * q2;
  const float um = fmaxf(fmaxf(u1.v.x, u1.v.y), fmaxf(u2.v.x, u2.v.y));
  if (um < LogMeanEps<float>::v) {
    L1 = f2(0.5f) * s1 * series_invF(u1);
    iL2 = f2(2.0f) * series_F(u2) * rs2;
  } else {
    float l1x, l1y, i2x, i2y;
    logmean_pair(a1.v.x, b1.v.x, a2.v.x, b2.v.x, l1x, i2x);
    logmean_pair(a1.v.y, b1.v.y, a2.v.y, b2.v.y, l1y, i2y);
    L1 = f2(l1x, l1y);
    iL2 = f2(i2x, i2y);
  }
}

}  // namespace crk
