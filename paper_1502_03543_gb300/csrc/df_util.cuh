// df_util.cuh -- double-float arithmetic on the FP32 pipes: a value is an
// unevaluated pair hi + lo of FP32 numbers (about 48 significant bits).
// Products of an FP32 number with a pair use the FMA residual (exact), sums
// use Knuth's TwoSum (exact), and a pair is widened into an FP64 accumulator
// by the integer-pipe widening of pdas_internal.cuh (exact).
#pragma once

#include "pdas_internal.cuh"

namespace pdas {

// (hi, lo) += a (vh + vl)
__device__ __forceinline__ void df_madd(float& hi, float& lo, float a, float vh, float vl) {
  const float ph = a * vh;
  const float pl = fmaf(a, vl, fmaf(a, vh, -ph));
  const float t = hi + ph;
  const float bb = t - hi;
  lo += ((hi - (t - bb)) + (ph - bb)) + pl;
  hi = t;
}

__device__ __forceinline__ void df_flush(double& acc, float& hi, float& lo) {
  acc += widen_bits(__float_as_uint(hi)) + widen_bits(__float_as_uint(lo));
  hi = 0.f;
  lo = 0.f;
}

// v -> (hi, lo) with hi = fl32(v), lo = fl32(v - hi).
__device__ __forceinline__ float2 df_split(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

}  // namespace pdas

namespace pdas {

// A double-float number as a value type, for the templates of the tile
// Cholesky (the FP64 tier of the mixed forms): hi + lo, |lo| <= ulp(hi) / 2.
// Sums use Knuth's TwoSum, products the FMA residual; about 14 FP32
// operations per multiply-add, ~46 significant bits.  The type and its
// operations live in a namespace of their own, so they are found by
// argument-dependent lookup only and hide no float or double overload.
namespace dfns {

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ explicit constexpr dfloat(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ dfloat df_renorm(float s, float t) {
  const float h = s + t;
  return dfloat(h, t - (h - s));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  const float s = a.hi + b.hi, bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  return df_renorm(s, e + a.lo + b.lo);
}
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
// a b + c
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);            // a.hi b.hi = p + e exactly
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  const float s = p + c.hi, bb = s - p;      // TwoSum(p, c.hi)
  const float t = (p - (s - bb)) + (c.hi - bb);
  return df_renorm(s, t + e + c.lo);
}
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) { return fma(a, b, dfloat(0)); }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }
__device__ __forceinline__ bool isfinite(dfloat a) { return ::isfinite(a.hi); }
__device__ __forceinline__ bool operator>(dfloat a, dfloat b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ dfloat __shfl_sync(unsigned mask, dfloat v, int src, int width = 32) {
  return dfloat(::__shfl_sync(mask, v.hi, src, width), ::__shfl_sync(mask, v.lo, src, width));
}
// 1 / sqrt(d): the FP32 estimate refined by one Newton step in double-float.
__device__ __forceinline__ dfloat inv_sqrt(dfloat d) {
  const float r0 = rsqrtf(d.hi);
  const dfloat r(r0, 0.f);
  const dfloat y = fma(d * r, r, dfloat(-1));  // d r^2 - 1
  return fma(dfloat(-0.5f * r0, 0.f), y, r);   // r (1 - y / 2)
}
__device__ __forceinline__ double df_to_double(dfloat a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfloat df_from_double(double v) {
  const float h = (float)v;
  return dfloat(h, (float)(v - (double)h));
}

}  // namespace dfns

using dfns::dfloat;
using dfns::df_from_double;
using dfns::df_to_double;

}  // namespace pdas
