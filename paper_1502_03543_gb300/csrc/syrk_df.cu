// syrk_df.cu -- the normal matrix M = A D A' (Section V) in double-float
// arithmetic on the FP32 pipes, for the FP64 tier of the mixed forms when A
// is exact in FP32 (stored as BF16 or FP32).
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so a pair of FP32 numbers
// (hi + lo, ~48-bit significand) is the cheaper way to FP64-grade sums:
//   D_j     = dh_j + dl_j                      (FP32 pair, precomputed);
//   B_qj    = A_qj D_j = bh + bl               (A_qj dh_j exact by FMA, plus A_qj dl_j);
//   M_pq    = sum_j A_pj (bh + bl)_qj          (A_pj bh_qj exact by FMA; the running sum
//                                                kept as hi + lo with Knuth's TwoSum);
// about 11 FP32 operations per term against one FP64 fused multiply-add.
// The sum is written as hi + lo in FP64.  128 x 128 lower-triangle tiles,
// 512 threads of 4 x 8 outputs (thread (tx, ty): rows ty + 32 i, columns
// tx + 16 j), so the 64 accumulator pairs of a thread stay in registers and
// 16 warps per SM hide the latency of the TwoSum chains.
#include "tile_core.cuh"

namespace pdas {

namespace {

__device__ __forceinline__ float as_f32(float v) { return v; }
__device__ __forceinline__ float as_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

__global__ void k_split_d(int64_t n, const double* __restrict__ D, float2* __restrict__ D2) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double d = D[j];
    const float h = (float)d;
    D2[j] = make_float2(h, (float)(d - (double)h));
  }
}

struct DfSmem {
  float a[kKc][kBig + 1];
  float bh[kKc][kBig + 1];
  float bl[kKc][kBig + 1];
};

constexpr int kDfThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kDfThreads, 1) k_syrk_df(int64_t m, int64_t n, const T* __restrict__ A,
                                                           const float2* __restrict__ D2, double* __restrict__ M,
                                                           int64_t ldm, const Scalars* sc) {
  __shared__ DfSmem sm;
  if (*(volatile const int*)&sc->status != 0) return;
  int64_t ti, tj;
  lower_tile(blockIdx.x, ti, tj);
  const int64_t p0 = ti * kBig, q0 = tj * kBig;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  constexpr int PER = (kBig * kKc) / kDfThreads;
  float hi[4][8], lo[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) hi[i][j] = lo[i][j] = 0.f;
  for (int64_t k0 = 0; k0 < n; k0 += kKc) {
    __syncthreads();
#pragma unroll
    for (int e4 = 0; e4 < PER; ++e4) {
      const int e = tid + e4 * kDfThreads;
      const int r = e / kKc, kk = e % kKc;
      const int64_t k = k0 + kk;
      const bool kin = k < n;
      sm.a[kk][r] = (kin && p0 + r < m) ? as_f32(A[(p0 + r) * n + k]) : 0.f;
      const float q = (kin && q0 + r < m) ? as_f32(A[(q0 + r) * n + k]) : 0.f;
      const float2 d = kin ? __ldg(D2 + k) : make_float2(0.f, 0.f);
      // B = A_q D as hi + lo: A dh exactly (product and its FMA residual), plus A dl
      const float ph = q * d.x;
      const float pl = fmaf(q, d.y, fmaf(q, d.x, -ph));
      const float s = ph + pl;
      sm.bh[kk][r] = s;
      sm.bl[kk][r] = pl - (s - ph);
    }
    __syncthreads();
#pragma unroll 1
    for (int kk = 0; kk < kKc; ++kk) {
      float a[4], bh[8], bl[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sm.a[kk][ty + 32 * i];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        bh[j] = sm.bh[kk][tx + 16 * j];
        bl[j] = sm.bl[kk][tx + 16 * j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float ph = a[i] * bh[j];
          const float pe = fmaf(a[i], bh[j], -ph);  // a bh = ph + pe exactly
          const float s = hi[i][j] + ph;            // TwoSum(hi, ph)
          const float bb = s - hi[i][j];
          const float err = (hi[i][j] - (s - bb)) + (ph - bb);
          hi[i][j] = s;
          lo[i][j] += err + fmaf(a[i], bl[j], pe);
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t p = p0 + ty + 32 * i;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t q = q0 + tx + 16 * j;
      if (p < m && q <= p) M[p * ldm + q] = (double)hi[i][j] + (double)lo[i][j];
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_syrk_df(cudaStream_t st, int64_t m, int64_t n, const T* A, const double* D, float2* D2,
                           double* M64, int64_t ldm, const Scalars* sc) {
  const int64_t g = (n + 255) / 256;
  k_split_d<<<(unsigned)(g < 1184 ? g : 1184), 256, 0, st>>>(n, D, D2);
  const int64_t tb = (m + kBig - 1) / kBig;
  k_syrk_df<T><<<(unsigned)(tb * (tb + 1) / 2), kDfThreads, 0, st>>>(m, n, A, D2, M64, ldm, sc);
  return cudaGetLastError();
}

template cudaError_t launch_syrk_df<float>(cudaStream_t, int64_t, int64_t, const float*, const double*, float2*,
                                           double*, int64_t, const Scalars*);
template cudaError_t launch_syrk_df<__nv_bfloat16>(cudaStream_t, int64_t, int64_t, const __nv_bfloat16*,
                                                   const double*, float2*, double*, int64_t, const Scalars*);

}  // namespace pdas
