// pond_packed.cuh -- two FP32 lanes per register pair for the mixed path
// (sm_103a).  Blackwell's paired FP32 instructions (fma.rn.f32x2 and its add
// and multiply, __ffma2_rn etc.) do the arithmetic of two independent values
// in one instruction.  The frame changes and syntheses of two stencil cells
// with the same face frame (their own shifts, shared synthesis constants)
// are such pairs, so the templated Hermite algebra of pond_hermite.cuh runs
// on this type unchanged, two cells at a time.  Each lane rounds exactly as
// the scalar FP32 operation does.
#pragma once
#include <cuda_runtime.h>

// The type and its operations live in a namespace of their own: the scalar
// code of namespace pond calls the global fma() unqualified, and the packed
// overloads are found by argument-dependent lookup.
namespace pond_pk {

struct f2 {
  float2 v;
  f2() = default;
  __device__ __forceinline__ f2(float2 a) : v(a) {}
  __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit f2(double a) : v(make_float2((float)a, (float)a)) {}
  __device__ __forceinline__ explicit f2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ explicit f2(int a) : v(make_float2((float)a, (float)a)) {}
  __device__ __forceinline__ float lo() const { return v.x; }
  __device__ __forceinline__ float hi() const { return v.y; }
};
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator-(f2 a) { return f2(-a.v.x, -a.v.y); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return a + (-b); }

}  // namespace pond_pk

namespace pond {
using pond_pk::f2;

// lane k of the result takes lane (bit ? lo : hi) of each member
__device__ __forceinline__ float pick(bool lo_lane, f2 a) { return lo_lane ? a.v.x : a.v.y; }
__device__ __forceinline__ DShift<f2> pick_rows(bool ua, bool ub, const DShift<f2> &C) {
  DShift<f2> R;
  R.d = f2(pick(ua, C.d), pick(ub, C.d)); R.d2 = f2(pick(ua, C.d2), pick(ub, C.d2));
  R.d3 = f2(pick(ua, C.d3), pick(ub, C.d3)); R.g2 = f2(pick(ua, C.g2), pick(ub, C.g2));
  R.g2x3 = f2(pick(ua, C.g2x3), pick(ub, C.g2x3)); R.g3 = f2(pick(ua, C.g3), pick(ub, C.g3));
  R.d4 = f2(pick(ua, C.d4), pick(ub, C.d4)); R.g2x6 = f2(pick(ua, C.g2x6), pick(ub, C.g2x6));
  R.g3x4 = f2(pick(ua, C.g3x4), pick(ub, C.g3x4)); R.g4 = f2(pick(ua, C.g4), pick(ub, C.g4));
  return R;
}
__device__ __forceinline__ DShift<float> pick_row(bool u, const DShift<f2> &C) {
  DShift<float> R;
  R.d = pick(u, C.d); R.d2 = pick(u, C.d2); R.d3 = pick(u, C.d3); R.g2 = pick(u, C.g2);
  R.g2x3 = pick(u, C.g2x3); R.g3 = pick(u, C.g3); R.d4 = pick(u, C.d4); R.g2x6 = pick(u, C.g2x6);
  R.g3x4 = pick(u, C.g3x4); R.g4 = pick(u, C.g4);
  return R;
}

}  // namespace pond
