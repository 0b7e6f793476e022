// Device helpers of the particle kernels (2D and 3D): the quadratic
// B-spline shape of a coordinate on its nearest node, the conversion-free
// nearest node, the 4-node Esirkepov window and small arithmetic helpers.
#pragma once

#include "common.cuh"

namespace pic {

template <typename R>
__device__ __forceinline__ R below(R v);
template <>
__device__ __forceinline__ float below<float>(float v) {
  return __int_as_float(__float_as_int(v) - 1);
}
template <>
__device__ __forceinline__ double below<double>(double v) {
  return __longlong_as_double(__double_as_longlong(v) - 1);
}

__device__ __forceinline__ float rsq(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsq(double v) { return rsqrt(v); }
__device__ __forceinline__ float quot(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double quot(double a, double b) { return a / b; }

// Nearest integer of v (|v| < 2^22 for float, 2^51 for double) and v minus
// it, without float-to-integer conversion instructions: adding 1.5 * 2^23
// (2^52) rounds v to an integer held in the low mantissa bits.  A tie
// (v = k + 1/2) may go to either neighbour; the quadratic shape has the same
// weights on both node sets there.
__device__ __forceinline__ int nearest(float v, float &d) {
  const float t = v + 12582912.0f;
  d = v - (t - 12582912.0f);
  return __float_as_int(t) - 0x4B400000;
}
__device__ __forceinline__ int nearest(double v, double &d) {
  const double t = v + 6755399441055744.0;
  d = v - (t - 6755399441055744.0);
  return (int)(__double_as_longlong(t) - 0x4338000000000000ll);
}

// Quadratic B-spline weights of the nodes i0-1, i0, i0+1 for offset d of a
// coordinate from its nearest node i0 (|d| <= 1/2).
template <typename R>
__device__ __forceinline__ void bspline(R d, R S[3]) {
  const R a = R(0.5) - d, b = R(0.5) + d;
  S[0] = R(0.5) * a * a;
  S[1] = R(0.75) - d * d;
  S[2] = R(0.5) * b * b;
}

// Primal (node) and dual (half-node) stencils of one coordinate xi (cells):
// ip = nearest node of xi, id = nearest node of xi - 1/2.
template <typename R>
__device__ __forceinline__ void shapes(R xi, int &ip, R Sp[3], int &id, R Sd[3]) {
  R dp, dd;
  ip = nearest(xi, dp);
  id = nearest(xi - R(0.5), dd);
  bspline(dp, Sp);
  bspline(dd, Sd);
}

template <typename R>
__device__ __forceinline__ int shape_primal(R xi, R S[3]) {
  R d;
  const int i = nearest(xi, d);
  bspline(d, S);
  return i;
}

// FP32 fixed-point current tiles: adding 1.5 * 2^23 to a value |v| < 2^22
// leaves round(v) (to nearest even) in the low mantissa bits, so one FMA
// both forms a contribution (already in the tile's unit) and rounds it, with
// no conversion instruction; red_fixed adds the rounded value of t = v +
// 1.5 * 2^23 into the 32-bit integer at shared address addr.
constexpr float kRoundMagic = 12582912.0f;
constexpr int kRoundBits = 0x4B400000;
__device__ __forceinline__ void red_fixed(uint32_t addr, float t) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(addr), "r"(__float_as_int(t) - kRoundBits));
}

// Place three shape weights in a 4-node window, shifted one node when sh.
template <typename R>
__device__ __forceinline__ void window4(const R S3[3], bool sh, R S[4]) {
  S[0] = sh ? R(0) : S3[0];
  S[1] = sh ? S3[0] : S3[1];
  S[2] = sh ? S3[1] : S3[2];
  S[3] = sh ? S3[2] : R(0);
}

}  // namespace pic
