// tile_core.cuh -- 64 x 64 rank-K tile product on the SIMT pipes, used by the
// FP64 / FP32 normal-matrix builder (M = A D A', Section V) and by the
// trailing update of the blocked Cholesky.
//
//   acc[i][j] += sum_k  P[p0 + r_i][k] * (D[k] if D) * Q[q0 + c_j][k]
//
// with r_i = ty + 16 i, c_j = tx + 16 j (tx = tid % 16, ty = tid / 16), so
// shared-memory reads are broadcasts (P) or consecutive (Q).  Rows outside
// [0, rows) contribute zeros.  256 threads; K is consumed in chunks of 16.
#pragma once

#include "pdas_internal.cuh"

namespace pdas {

constexpr int kKc = 16;

template <typename TIn, typename TAcc>
struct TileSmem {
  TAcc p[kKc][kTile + 1];
  TAcc q[kKc][kTile + 1];
};

template <typename TAcc>
__device__ __forceinline__ TAcc to_acc(double v);
template <>
__device__ __forceinline__ double to_acc<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_acc<float>(double v) { return (float)v; }

// Loads element (row, k) of a row-major operand as TAcc; scaled by D[k] when D
// is given (the product A_pk D_k is formed in FP64, then rounded to TAcc).
template <typename TIn, typename TAcc>
__device__ __forceinline__ TAcc load_op(const TIn* X, int64_t ld, int64_t row, int64_t k, const double* D) {
  const double v = widen(X[row * ld + k]);
  return to_acc<TAcc>(D ? v * __ldg(D + k) : v);
}

template <typename TIn, typename TAcc>
__device__ void tile_rank_k(const TIn* __restrict__ P, int64_t ldp, int64_t p0, int64_t prows,
                            const TIn* __restrict__ Q, int64_t ldq, int64_t q0, int64_t qrows, int64_t K,
                            const double* __restrict__ D, TileSmem<TIn, TAcc>& sm, TAcc (&acc)[4][4]) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  for (int64_t k0 = 0; k0 < K; k0 += kKc) {
    __syncthreads();
#pragma unroll
    for (int e4 = 0; e4 < (kTile * kKc) / kThreads; ++e4) {
      const int e = tid + e4 * kThreads;
      const int r = e / kKc, kk = e % kKc;
      const int64_t k = k0 + kk;
      const bool kin = k < K;
      sm.p[kk][r] = (kin && p0 + r < prows) ? load_op<TIn, TAcc>(P, ldp, p0 + r, k, D) : TAcc(0);
      sm.q[kk][r] = (kin && q0 + r < qrows) ? load_op<TIn, TAcc>(Q, ldq, q0 + r, k, nullptr) : TAcc(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kKc; ++kk) {
      TAcc a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sm.p[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sm.q[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
}

// ---- 128 x 128 tiles, 8 x 8 outputs per thread ---------------------------
// Same product as tile_rank_k on a 128 x 128 tile: thread (tx, ty) owns rows
// ty + 16 i and columns tx + 16 j (i, j < 8).  The next K chunk is fetched
// into registers while the current one is multiplied.
constexpr int kBig = 128;
static_assert(kBig == kCholTile, "the tile Cholesky works on 128 x 128 tiles");

template <typename TAcc>
struct TileSmem128 {
  TAcc p[kKc][kBig + 1];
  TAcc q[kKc][kBig + 1];
};

template <typename TIn, typename TAcc>
__device__ void tile128_rank_k(const TIn* __restrict__ P, int64_t ldp, int64_t p0, int64_t prows,
                               const TIn* __restrict__ Q, int64_t ldq, int64_t q0, int64_t qrows, int64_t K,
                               const double* __restrict__ D, TileSmem128<TAcc>& sm, TAcc (&acc)[8][8]) {
  constexpr int PER = (kBig * kKc) / kThreads;  // elements of each operand per thread per chunk
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  TAcc rp[PER], rq[PER];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int e4 = 0; e4 < PER; ++e4) {
      const int e = tid + e4 * kThreads;
      const int r = e / kKc, kk = e % kKc;
      const int64_t k = k0 + kk;
      const bool kin = k < K;
      rp[e4] = (kin && p0 + r < prows) ? load_op<TIn, TAcc>(P, ldp, p0 + r, k, D) : TAcc(0);
      rq[e4] = (kin && q0 + r < qrows) ? load_op<TIn, TAcc>(Q, ldq, q0 + r, k, nullptr) : TAcc(0);
    }
  };
  fetch(0);
  for (int64_t k0 = 0; k0 < K; k0 += kKc) {
    __syncthreads();
#pragma unroll
    for (int e4 = 0; e4 < PER; ++e4) {
      const int e = tid + e4 * kThreads;
      sm.p[e % kKc][e / kKc] = rp[e4];
      sm.q[e % kKc][e / kKc] = rq[e4];
    }
    __syncthreads();
    if (k0 + kKc < K) fetch(k0 + kKc);
#pragma unroll
    for (int kk = 0; kk < kKc; ++kk) {
      TAcc a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = sm.p[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = sm.q[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
}

// Lower-triangle tile index t -> (ti, tj) with ti >= tj.
__device__ __forceinline__ void lower_tile(int64_t t, int64_t& ti, int64_t& tj) {
  int64_t i = (int64_t)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);  // FP32 estimate, corrected below
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  ti = i;
  tj = t - i * (i + 1) / 2;
}

}  // namespace pdas
