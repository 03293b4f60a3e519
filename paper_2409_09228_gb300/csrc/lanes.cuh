// Lane types for the fused kernel: float (one track per thread), F2 (two
// tracks per thread, held in the two halves of a float2), and double (the
// FP64 variant, one track per thread, IEEE operations throughout).
//
// The per-track math is written once as templates over the lane type.  With
// F2 every add, multiply and fused multiply-add is one packed sm_100+
// instruction (__fadd2_rn / __fmul2_rn / __ffma2_rn, each component rounded
// exactly like the scalar operation), so one issue slot carries the FP32 work
// of two tracks; loads and stores become 64-bit.  Operations without a packed
// form (reciprocal, rsqrt, comparisons) run per component.  Comparisons give
// masks (bool or M2) that all()/any()/sel() consume.
#pragma once

#include <cuda_runtime.h>

namespace fitk {

struct F2 {
  float2 v;
  __device__ __forceinline__ F2() {}
  __device__ __forceinline__ F2(float a) : v(make_float2(a, a)) {}  // broadcast
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit F2(float2 a) : v(a) {}
};

struct M2 {
  bool x, y;
};

// ---- arithmetic ----------------------------------------------------------
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__fadd2_rn(a.v, (-b).v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }
__device__ __forceinline__ F2& operator*=(F2& a, F2 b) { return a = a * b; }

__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

// Division and square root where a couple of ulp are far below the fit's
// tolerance: the approximate reciprocal, square root and rsqrt (MUFU) instead
// of the IEEE sequences.
__device__ __forceinline__ float frcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ F2 frcp(F2 x) { return F2(frcp(x.v.x), frcp(x.v.y)); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
// a * (1/b): the reciprocals per lane, the product packed
__device__ __forceinline__ F2 fdiv(F2 a, F2 b) { return a * frcp(b); }
// Approximate square root and reciprocal square root (one MUFU operation
// each, relative error ~2^-23); NaN for x < 0, which every caller either
// excludes by its own test or sends down a failing branch.  Subnormal
// inputs flush to zero (.ftz): the fit's quantities are far from 1e-38, and
// the subnormal-safe forms cost a test and two multiplies around each MUFU.
__device__ __forceinline__ float fsqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ F2 fsqrt(F2 x) { return F2(fsqrt(x.v.x), fsqrt(x.v.y)); }
__device__ __forceinline__ float frsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ F2 frsqrt(F2 x) { return F2(frsqrt(x.v.x), frsqrt(x.v.y)); }
__device__ __forceinline__ float fabs_(float x) { return fabsf(x); }
__device__ __forceinline__ F2 fabs_(F2 x) { return F2(fabsf(x.v.x), fabsf(x.v.y)); }
__device__ __forceinline__ float fmax_(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ F2 fmax_(F2 a, F2 b) { return F2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y)); }
__device__ __forceinline__ float floor_(float x) { return floorf(x); }
__device__ __forceinline__ F2 floor_(F2 x) { return F2(floorf(x.v.x), floorf(x.v.y)); }
__device__ __forceinline__ float copysign_(float a, float b) { return copysignf(a, b); }
__device__ __forceinline__ F2 copysign_(F2 a, F2 b) {
  return F2(copysignf(a.v.x, b.v.x), copysignf(a.v.y, b.v.y));
}

// ---- masks ---------------------------------------------------------------
__device__ __forceinline__ bool le(float a, float b) { return a <= b; }
__device__ __forceinline__ M2 le(F2 a, F2 b) { return {a.v.x <= b.v.x, a.v.y <= b.v.y}; }
__device__ __forceinline__ bool lt(float a, float b) { return a < b; }
__device__ __forceinline__ M2 lt(F2 a, F2 b) { return {a.v.x < b.v.x, a.v.y < b.v.y}; }
__device__ __forceinline__ bool finite_(float a) { return isfinite(a); }
__device__ __forceinline__ M2 finite_(F2 a) { return {(bool)isfinite(a.v.x), (bool)isfinite(a.v.y)}; }
__device__ __forceinline__ bool all(bool m) { return m; }
__device__ __forceinline__ bool all(M2 m) { return m.x && m.y; }
__device__ __forceinline__ bool any(bool m) { return m; }
__device__ __forceinline__ bool any(M2 m) { return m.x || m.y; }
__device__ __forceinline__ bool not_(bool m) { return !m; }
__device__ __forceinline__ M2 not_(M2 m) { return {!m.x, !m.y}; }
__device__ __forceinline__ bool and_(bool a, bool b) { return a && b; }
__device__ __forceinline__ M2 and_(M2 a, M2 b) { return {a.x && b.x, a.y && b.y}; }
__device__ __forceinline__ bool or_(bool a, bool b) { return a || b; }
__device__ __forceinline__ M2 or_(M2 a, M2 b) { return {a.x || b.x, a.y || b.y}; }
__device__ __forceinline__ float sel(bool m, float a, float b) { return m ? a : b; }
__device__ __forceinline__ F2 sel(M2 m, F2 a, F2 b) {
  return F2(m.x ? a.v.x : b.v.x, m.y ? a.v.y : b.v.y);
}

// ---- double (the FP64 variant, one track per thread): IEEE operations ------
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }
__device__ __forceinline__ double fsqrt(double x) { return ::sqrt(x); }  // NaN for x < 0, as in FP32
__device__ __forceinline__ double frsqrt(double x) { return 1.0 / ::sqrt(x); }
__device__ __forceinline__ double fabs_(double x) { return ::fabs(x); }
__device__ __forceinline__ double floor_(double x) { return ::floor(x); }
__device__ __forceinline__ double fmax_(double a, double b) { return ::fmax(a, b); }
__device__ __forceinline__ double copysign_(double a, double b) { return ::copysign(a, b); }
__device__ __forceinline__ bool le(double a, double b) { return a <= b; }
__device__ __forceinline__ bool lt(double a, double b) { return a < b; }
__device__ __forceinline__ bool finite_(double a) { return isfinite(a); }
__device__ __forceinline__ double sel(bool m, double a, double b) { return m ? a : b; }

// ---- lanes ---------------------------------------------------------------
template <class T>
struct Lanes;
template <>
struct Lanes<float> {
  static constexpr int n = 1;
  using M = bool;
  __device__ __forceinline__ static float get(float a, int) { return a; }
  __device__ __forceinline__ static bool get(bool m, int) { return m; }
};
template <>
struct Lanes<double> {
  static constexpr int n = 1;
  using M = bool;
  __device__ __forceinline__ static double get(double a, int) { return a; }
  __device__ __forceinline__ static bool get(bool m, int) { return m; }
};
template <>
struct Lanes<F2> {
  static constexpr int n = 2;
  using M = M2;
  __device__ __forceinline__ static float get(F2 a, int i) { return i ? a.v.y : a.v.x; }
  __device__ __forceinline__ static bool get(M2 m, int i) { return i ? m.y : m.x; }
};

// Streaming loads and stores of lane-consecutive tracks (p points at the
// first track; for F2 it is 8-byte aligned).
__device__ __forceinline__ void ld(float& d, const float* p) { d = __ldcs(p); }
__device__ __forceinline__ void ld(F2& d, const float* p) {
  d = F2(__ldcs(reinterpret_cast<const float2*>(p)));
}
__device__ __forceinline__ void ld(double& d, const double* p) { d = __ldcs(p); }
__device__ __forceinline__ void st(double* p, double v) { *p = v; }
__device__ __forceinline__ void st(float* p, float v) { *p = v; }
__device__ __forceinline__ void st(float* p, F2 v) { *reinterpret_cast<float2*>(p) = v.v; }

}  // namespace fitk
