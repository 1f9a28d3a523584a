// gemv_df.cu -- the passes over A of the mixed forms (the right-hand side
// r = A x and the refinement products A(D(A' v)) of Section V, and
// ds = -A' dy) in double-float arithmetic on the FP32 pipes, for A stored as
// FP32 or BF16 (every entry exact in FP32).
//
// GB300 issues FP64 at 1/64 of its FP32 rate, so an FP64 multiply-add per
// entry of A makes each pass compute-bound at about 5x the time it takes to
// stream A from HBM.  Here the vector is first split into FP32 pairs
// v = vh + vl (|vl| <= 2^-24 |vh|, 48 significant bits), and each term is
//   a vh = ph + pe        exactly (FMA residual),
//   a v  ~ ph + (pe + a vl)        (relative error <= 2^-47),
// summed into an FP32 pair with Knuth's TwoSum on the high part; every 16 or
// 32 terms the pair is widened exactly (integer pipes) into an FP64
// accumulator.  About 10 FP32 operations per entry against one FP64
// multiply-add; the error stays within a few units of 2^-44 of sum |a v|,
// the level of FP64 accumulation over the same row length.  Block
// reductions, chunk sums and the norm slots are FP64, as in the FP64 passes.
#include "df_util.cuh"
#include "reduce_util.cuh"

namespace pdas {

namespace {

template <typename T>
struct Vec32;
template <>
struct Vec32<float> {
  static constexpr int N = 4;
  __device__ static void load(const float* p, float* o) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  __device__ static float one(const float* p) { return __ldg(p); }
};
template <>
struct Vec32<__nv_bfloat16> {
  static constexpr int N = 8;
  __device__ static void load(const __nv_bfloat16* p, float* o) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[2 * i] = __uint_as_float(w[i] << 16);
      o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
  __device__ static float one(const __nv_bfloat16* p) { return __bfloat162float(*p); }
};

__global__ void k_split_pairs(int64_t n, const double* __restrict__ v, float2* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = df_split(v[j]);
}

// out_p = A_p. v (base == null) or base_p - A_p. v; ROWS rows per block; as
// k_gemv, with the norm slots.
template <typename T, int ROWS>
__global__ void __launch_bounds__(kThreads) k_gemv_df(int64_t m, int64_t n, const T* __restrict__ A,
                                                      const float2* __restrict__ v2, const double* __restrict__ base,
                                                      double* __restrict__ out, int vec_ok, double* part,
                                                      unsigned* tickets, Scalars* sc, int norm_slot) {
  __shared__ double sm[32];
  __shared__ double rowsum[ROWS];
  if (failed(sc)) return;
  constexpr int VN = Vec32<T>::N;
  const int64_t p0 = (int64_t)blockIdx.x * ROWS;
  double acc[ROWS];
  float hi[ROWS], lo[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    acc[r] = 0.0;
    hi[r] = lo[r] = 0.f;
  }
  if (vec_ok) {
    int it = 0;
    for (int64_t j = (int64_t)threadIdx.x * VN; j < n; j += (int64_t)blockDim.x * VN) {
      float vh[VN], vl[VN];
#pragma unroll
      for (int k = 0; k < VN; k += 2) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(v2 + j + k));
        vh[k] = q.x; vl[k] = q.y; vh[k + 1] = q.z; vl[k + 1] = q.w;
      }
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        if (p0 + r < m) {
          float a[VN];
          Vec32<T>::load(A + (p0 + r) * n + j, a);
#pragma unroll
          for (int k = 0; k < VN; ++k) df_madd(hi[r], lo[r], a[k], vh[k], vl[k]);
        }
      }
      if ((++it & 3) == 0) {
#pragma unroll
        for (int r = 0; r < ROWS; ++r) df_flush(acc[r], hi[r], lo[r]);
      }
    }
  } else {
    int it = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const float2 q = __ldg(v2 + j);
#pragma unroll
      for (int r = 0; r < ROWS; ++r)
        if (p0 + r < m) df_madd(hi[r], lo[r], Vec32<T>::one(A + (p0 + r) * n + j), q.x, q.y);
      if ((++it & 15) == 0) {
#pragma unroll
        for (int r = 0; r < ROWS; ++r) df_flush(acc[r], hi[r], lo[r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < ROWS; ++r) df_flush(acc[r], hi[r], lo[r]);
  double amax = 0.0;
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const double t = block_reduce<0>(acc[r], sm);
    if (threadIdx.x == 0) rowsum[r] = t;
  }
  __syncthreads();
  if (threadIdx.x < ROWS && p0 + threadIdx.x < m) {
    const int64_t p = p0 + threadIdx.x;
    const double o = base ? base[p] - rowsum[threadIdx.x] : rowsum[threadIdx.x];
    out[p] = o;
    amax = fabs(o);
    if (!isfinite(o)) amax = INFINITY;
  }
  if (norm_slot < 0) return;
  const double bm = block_reduce<1>(amax, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = bm;
  if (!last_block(tickets + T_NORM)) return;
  const double g = combine<1>(part, gridDim.x, sm);
  if (threadIdx.x == 0) {
    if (norm_slot == 0) sc->rnorm = g; else sc->rho_norm = g;
    tickets[T_NORM] = 0;
  }
}

// Partial column sums part[c][j] = sum_{p in chunk c} A_pj u_p, as
// k_gemv_t_part; the chunk sum is finished by k_gemv_t_finish in FP64.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_gemv_t_part_df(int64_t m, int64_t n, const T* __restrict__ A,
                                                             const float2* __restrict__ u2, double* __restrict__ part,
                                                             int64_t rows_per_chunk, int vec_ok) {
  constexpr int VN = Vec32<T>::N;
  const int64_t pbeg = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t pend = pbeg + rows_per_chunk < m ? pbeg + rows_per_chunk : m;
  double* dst = part + (int64_t)blockIdx.y * n;
  if (vec_ok) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VN;
    if (j >= n) return;
    double acc[VN];
    float hi[VN], lo[VN];
#pragma unroll
    for (int k = 0; k < VN; ++k) {
      acc[k] = 0.0;
      hi[k] = lo[k] = 0.f;
    }
    int it = 0;
#pragma unroll 4
    for (int64_t p = pbeg; p < pend; ++p) {
      float a[VN];
      Vec32<T>::load(A + p * n + j, a);
      const float2 q = __ldg(u2 + p);
#pragma unroll
      for (int k = 0; k < VN; ++k) df_madd(hi[k], lo[k], a[k], q.x, q.y);
      if ((++it & 15) == 0) {
#pragma unroll
        for (int k = 0; k < VN; ++k) df_flush(acc[k], hi[k], lo[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < VN; ++k) {
      df_flush(acc[k], hi[k], lo[k]);
      dst[j + k] = acc[k];
    }
  } else {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double acc = 0.0;
    float hi = 0.f, lo = 0.f;
    int it = 0;
    for (int64_t p = pbeg; p < pend; ++p) {
      const float2 q = __ldg(u2 + p);
      df_madd(hi, lo, Vec32<T>::one(A + p * n + j), q.x, q.y);
      if ((++it & 15) == 0) df_flush(acc, hi, lo);
    }
    df_flush(acc, hi, lo);
    dst[j] = acc;
  }
}

}  // namespace

cudaError_t launch_split_pairs(cudaStream_t st, int64_t n, const double* v, float2* out) {
  k_split_pairs<<<grid_for(n, 4), kThreads, 0, st>>>(n, v, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gemv_df(cudaStream_t st, int64_t m, int64_t n, const T* A, const float2* v2, const double* base,
                           double* out, double* part, unsigned* tickets, Scalars* sc, int norm_slot) {
  constexpr int ROWS = 4;
  const int64_t grid = (m + ROWS - 1) / ROWS;
  if (norm_slot >= 0 && grid > kPartMax) return cudaErrorInvalidConfiguration;
  k_gemv_df<T, ROWS><<<(unsigned)grid, kThreads, 0, st>>>(m, n, A, v2, base, out, vec_aligned(A, n) ? 1 : 0, part,
                                                            tickets, sc, norm_slot);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gemv_t_df(cudaStream_t st, int64_t m, int64_t n, const T* A, const float2* u2, double* part,
                             int chunks, int64_t rows_per_chunk) {
  const bool vok = vec_aligned(A, n);
  const int64_t cols_per_block = (int64_t)kThreads * (vok ? Vec32<T>::N : 1);
  dim3 grid((unsigned)((n + cols_per_block - 1) / cols_per_block), (unsigned)chunks);
  k_gemv_t_part_df<T><<<grid, kThreads, 0, st>>>(m, n, A, u2, part, rows_per_chunk, vok ? 1 : 0);
  return cudaGetLastError();
}

template cudaError_t launch_gemv_df<float>(cudaStream_t, int64_t, int64_t, const float*, const float2*, const double*,
                                           double*, double*, unsigned*, Scalars*, int);
template cudaError_t launch_gemv_df<__nv_bfloat16>(cudaStream_t, int64_t, int64_t, const __nv_bfloat16*,
                                                   const float2*, const double*, double*, double*, unsigned*,
                                                   Scalars*, int);
template cudaError_t launch_gemv_t_df<float>(cudaStream_t, int64_t, int64_t, const float*, const float2*, double*,
                                             int, int64_t);
template cudaError_t launch_gemv_t_df<__nv_bfloat16>(cudaStream_t, int64_t, int64_t, const __nv_bfloat16*,
                                                     const float2*, double*, int, int64_t);

}  // namespace pdas
