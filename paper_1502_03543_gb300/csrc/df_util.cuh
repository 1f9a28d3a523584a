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
