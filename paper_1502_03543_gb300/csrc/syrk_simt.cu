// syrk_simt.cu -- the normal matrix M = A D A' (Section V: the system
// (A D A') dy = A x) on the SIMT pipes: FP64 for the plain FP64 form and for
// the FP64 re-factorisation of the mixed forms, FP32 for the FP32_IR form.
// Only the lower triangle (p >= q) is formed and written.
#include "tile_core.cuh"

namespace pdas {

namespace {

template <typename T, typename TAcc>
__global__ void __launch_bounds__(kThreads) k_syrk_simt(int64_t m, int64_t n, const T* __restrict__ A,
                                                        const double* __restrict__ D, TAcc* __restrict__ M,
                                                        int64_t ldm, const Scalars* sc) {
  __shared__ TileSmem<T, TAcc> sm;
  if (*(volatile const int*)&sc->status != 0) return;
  int64_t ti, tj;
  lower_tile(blockIdx.x, ti, tj);
  const int64_t p0 = ti * kTile, q0 = tj * kTile;
  TAcc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = TAcc(0);
  // M_pq = sum_j (A_pj D_j) A_qj
  tile_rank_k<T, TAcc>(A, n, p0, m, A, n, q0, m, n, D, sm, acc);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t p = p0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t q = q0 + tx + 16 * j;
      if (p < m && q <= p) M[p * ldm + q] = acc[i][j];
    }
  }
}

// FP32 normal matrix on 128 x 128 tiles (8 x 8 per thread).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_syrk_simt128(int64_t m, int64_t n, const T* __restrict__ A,
                                                           const double* __restrict__ D, float* __restrict__ M,
                                                           int64_t ldm, const Scalars* sc) {
  __shared__ TileSmem128<float> sm;
  if (*(volatile const int*)&sc->status != 0) return;
  int64_t ti, tj;
  lower_tile(blockIdx.x, ti, tj);
  const int64_t p0 = ti * kBig, q0 = tj * kBig;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  tile128_rank_k<T, float>(A, n, p0, m, A, n, q0, m, n, D, sm, acc);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t p = p0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t q = q0 + tx + 16 * j;
      if (p < m && q <= p) M[p * ldm + q] = acc[i][j];
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_syrk_simt(cudaStream_t st, int64_t m, int64_t n, const T* A, const double* D, double* M64,
                             float* M32, int64_t ldm, const Scalars* sc) {
  const int64_t t = (m + kTile - 1) / kTile;
  const int64_t tiles = t * (t + 1) / 2;
  if (M64)
    k_syrk_simt<T, double><<<(unsigned)tiles, kThreads, 0, st>>>(m, n, A, D, M64, ldm, sc);
  else {
    const int64_t tb = (m + kBig - 1) / kBig;
    k_syrk_simt128<T><<<(unsigned)(tb * (tb + 1) / 2), kThreads, 0, st>>>(m, n, A, D, M32, ldm, sc);
  }
  return cudaGetLastError();
}

template cudaError_t launch_syrk_simt<double>(cudaStream_t, int64_t, int64_t, const double*, const double*, double*,
                                              float*, int64_t, const Scalars*);
template cudaError_t launch_syrk_simt<float>(cudaStream_t, int64_t, int64_t, const float*, const double*, double*,
                                             float*, int64_t, const Scalars*);
template cudaError_t launch_syrk_simt<__nv_bfloat16>(cudaStream_t, int64_t, int64_t, const __nv_bfloat16*,
                                                     const double*, double*, float*, int64_t, const Scalars*);

}  // namespace pdas
