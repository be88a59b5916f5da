// Two FP32 lanes in one register pair, computed with the packed FP32 instructions of sm_100 and
// later (__fadd2_rn, __fmul2_rn, __ffma2_rn: one instruction for both lanes, each lane rounded
// exactly as the scalar operation).  The paired 16-bit step holds node x in lane .x and node x+1
// in lane .y, which is also how the two nodes' 16-bit values of one direction share a 32-bit word,
// so the collision of Eqs. 15-17 and the stencils of Eq. 12 run once for the pair.
//
// The compiler contracts a scalar a*b + c into one FMA but does not form packed FMAs, so a
// product here is a proxy (F2Prod) that becomes __ffma2_rn when it meets an addition or
// subtraction and __fmul2_rn otherwise: the same contraction a scalar expression gets, written
// out.  Which of two products becomes the FMA in a*b + c*d may differ from the scalar kernel,
// so results agree with the one-node kernel to rounding, not bit for bit.
#pragma once
#include <cuda_runtime.h>

namespace lbmch {

struct F2 {
  float2 v;
  F2() = default;
  __host__ __device__ constexpr F2(float2 p) : v(p) {}
  __host__ __device__ constexpr F2(float s) : v{s, s} {}
  __host__ __device__ constexpr F2(double s) : v{(float)s, (float)s} {}
  __host__ __device__ constexpr F2(int s) : v{(float)s, (float)s} {}
  __host__ __device__ constexpr F2(float a, float b) : v{a, b} {}
};

__device__ __forceinline__ F2 f2_neg(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
// a - b in one instruction (the library has no packed subtraction).
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(d)
      : "l"(*reinterpret_cast<const unsigned long long*>(&a.v)), "l"(*reinterpret_cast<const unsigned long long*>(&b.v)));
  return F2(*reinterpret_cast<const float2*>(&d));
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

// a * b, not yet rounded.
struct F2Prod {
  F2 a, b;
  __device__ __forceinline__ operator F2() const { return f2_mul(a, b); }
};

__device__ __forceinline__ F2Prod operator*(F2 a, F2 b) { return {a, b}; }
__device__ __forceinline__ F2Prod operator*(F2Prod p, F2 b) { return {F2(p), b}; }
__device__ __forceinline__ F2Prod operator*(F2 a, F2Prod q) { return {a, F2(q)}; }
__device__ __forceinline__ F2Prod operator*(F2Prod p, F2Prod q) { return {F2(p), F2(q)}; }
__device__ __forceinline__ F2Prod operator-(F2Prod p) { return {f2_neg(p.a), p.b}; }
__device__ __forceinline__ F2 operator-(F2 a) { return f2_neg(a); }

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return f2_add(a, b); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return f2_sub(a, b); }
__device__ __forceinline__ F2 operator+(F2Prod p, F2 c) { return f2_fma(p.a, p.b, c); }
__device__ __forceinline__ F2 operator+(F2 c, F2Prod p) { return f2_fma(p.a, p.b, c); }
__device__ __forceinline__ F2 operator-(F2Prod p, F2 c) { return f2_fma(p.a, p.b, f2_neg(c)); }
__device__ __forceinline__ F2 operator-(F2 c, F2Prod p) { return f2_fma(f2_neg(p.a), p.b, c); }
__device__ __forceinline__ F2 operator+(F2Prod p, F2Prod q) { return f2_fma(p.a, p.b, F2(q)); }
__device__ __forceinline__ F2 operator-(F2Prod p, F2Prod q) { return f2_fma(p.a, p.b, f2_neg(F2(q))); }
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(a.v.x / b.v.x, a.v.y / b.v.y); }
__device__ __forceinline__ F2 operator/(F2Prod p, F2 b) { return F2(p) / b; }

// 1/x for the collision's runtime reciprocals (1/rho, the relaxation frequency): the hardware's
// approximate reciprocal of each lane (relative error below 2^-23) refined by one Newton-Raphson
// step r' = r + r (1 - x r), two packed FMAs, instead of two IEEE divisions.  The step squares
// the relative error, so r' is the correctly rounded 1/x or one unit of the last place from it.
__device__ __forceinline__ F2 recip(F2 x) {
  float rx, ry;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rx) : "f"(x.v.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ry) : "f"(x.v.y));
  const F2 r(rx, ry);
  const F2 e = f2_fma(f2_neg(x), r, F2(1.0f));
  return f2_fma(r, e, r);
}

__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator+=(F2& a, F2Prod p) { return a = a + p; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2Prod p) { return a = a - p; }

}  // namespace lbmch
