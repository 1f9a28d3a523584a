// trsv_blk.cu -- the two triangular solves of the normal equations with the
// FP32 factor of the mixed forms (Section V-A: L z = A x, then L' dy = z),
// in 128-row blocks.  The factor launch leaves U_b = L_bb^{-T} for every
// diagonal tile, so a block applies U_b' (forward) or U_b (backward) as a
// 128 x 128 product instead of a 128-step substitution; the dependency chain
// from block to block is then one tile product with the newest neighbour
// block and one with U_b.  The FP32 factor is a preconditioner here (the
// mixed forms refine in FP64 afterwards), so the explicit inverse of each
// diagonal tile is accurate enough; the plain FP64 form keeps substitution.
//
// One launch per solve.  Blocks take block rows in order from a ticket
// counter and wait (bounded, 2 s) for the flags of the blocks they depend
// on, which were handed out earlier: no deadlock.  Thread layout for the
// off-diagonal tiles: warp w holds rows 16 w .. 16 w + 15, lane l columns
// 4 l .. 4 l + 3 (16-byte loads along the rows); tiles are loaded before the
// wait for the block they multiply.
#include "sync_util.cuh"
#include "tile_core.cuh"

namespace pdas {

namespace {

struct TrsvSmem {
  float U[kBig][kBig + 1];  // U_b = L_bb^{-T}
  float rhs[kBig];
  float red[8][kBig];
  int b;
};

// 16 per-lane partial sums reduced across the warp by exchanging halves:
// lane l ends with the total of entry (l >> 1) & 15 (16 shuffles in all).
__device__ __forceinline__ float reduce16(float (&v)[16], int lane) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const bool up = lane & 16;
    const float keep = up ? v[k + 8] : v[k], send = up ? v[k] : v[k + 8];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool up = lane & 8;
    const float keep = up ? v[k + 4] : v[k], send = up ? v[k] : v[k + 4];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool up = lane & 4;
    const float keep = up ? v[k + 2] : v[k], send = up ? v[k] : v[k + 2];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool up = lane & 2;
    const float keep = up ? v[1] : v[0], send = up ? v[0] : v[1];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ void load_u(TrsvSmem& sm, const float* __restrict__ Ub) {
  for (int e = threadIdx.x; e < kBig * kBig; e += blockDim.x) sm.U[e >> 7][e & 127] = __ldg(Ub + e);
}

// L z = v: z_b = U_b' (v_b - sum_{j<b} L_bj z_j).
__global__ void __launch_bounds__(kThreads) k_trsv_lower_blk(int64_t m, int64_t ldm, const float* __restrict__ L,
                                                             const float* __restrict__ Uinv,
                                                             const double* __restrict__ v, double* z, int* flags,
                                                             unsigned* ticket, Scalars* sc) {
  extern __shared__ __align__(16) unsigned char trsv_blk_smem[];
  TrsvSmem& sm = *reinterpret_cast<TrsvSmem*>(trsv_blk_smem);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) sm.b = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  if (dev_failed(sc)) return;
  const int b = sm.b;
  const int64_t r0 = (int64_t)b * kBig;
  const int rb = (int)(m - r0 < kBig ? m - r0 : kBig);
  load_u(sm, Uinv + (int64_t)b * kBig * kBig);
  float part[16];
#pragma unroll
  for (int rr = 0; rr < 16; ++rr) part[rr] = 0.f;
  bool ok = true;
  for (int64_t j = 0; j < b; ++j) {  // tile j is full (j < b <= nb - 1)
    float4 lv[16];
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      const int64_t row = r0 + 16 * w + rr;
      lv[rr] = row < m ? __ldg(reinterpret_cast<const float4*>(L + row * ldm + j * kBig + 4 * lane))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    ok = warp_wait(flags, j, sc);
    if (!ok) break;
    const double* zj = z + j * kBig + 4 * lane;
    const float z0 = (float)__ldcg(zj), z1 = (float)__ldcg(zj + 1), z2 = (float)__ldcg(zj + 2),
                z3 = (float)__ldcg(zj + 3);
#pragma unroll
    for (int rr = 0; rr < 16; ++rr)
      part[rr] = fmaf(lv[rr].x, z0, fmaf(lv[rr].y, z1, fmaf(lv[rr].z, z2, fmaf(lv[rr].w, z3, part[rr]))));
  }
  const float tot = reduce16(part, lane);
  const int row = 16 * w + ((lane >> 1) & 15);
  if ((lane & 1) == 0) sm.rhs[row] = row < rb ? (float)v[r0 + row] - tot : 0.f;
  if (__syncthreads_or(!ok)) return;  // a wait gave up: the status says why
  const int c = tid & 127, h = tid >> 7;  // z_c = sum_r U_rc rhs_r, rows split in two halves
  float s = 0.f;
#pragma unroll 8
  for (int r = 64 * h; r < 64 * h + 64; ++r) s = fmaf(sm.U[r][c], sm.rhs[r], s);
  sm.red[h][c] = s;
  __syncthreads();
  if (tid < rb) z[r0 + tid] = (double)(sm.red[0][tid] + sm.red[1][tid]);
  __threadfence();
  __syncthreads();
  if (tid == 0) st_release(flags + b, 1);
}

// L' y = z: y_b = U_b (z_b - sum_{k>b} L_kb' y_k); blocks go from the last.
__global__ void __launch_bounds__(kThreads) k_trsv_upper_blk(int64_t m, int64_t ldm, const float* __restrict__ L,
                                                             const float* __restrict__ Uinv,
                                                             const double* __restrict__ zin, double* y, int* flags,
                                                             unsigned* ticket, Scalars* sc) {
  extern __shared__ __align__(16) unsigned char trsv_blk_smem[];
  TrsvSmem& sm = *reinterpret_cast<TrsvSmem*>(trsv_blk_smem);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t nblk = (m + kBig - 1) / kBig;
  if (tid == 0) sm.b = (int)(nblk - 1 - (int64_t)atomicAdd(ticket, 1u));
  __syncthreads();
  if (dev_failed(sc)) return;
  const int b = sm.b;
  const int64_t r0 = (int64_t)b * kBig;
  const int rb = (int)(m - r0 < kBig ? m - r0 : kBig);
  load_u(sm, Uinv + (int64_t)b * kBig * kBig);
  float colp[4] = {0.f, 0.f, 0.f, 0.f};  // columns 4 lane .. 4 lane + 3 of tile b, this warp's rows
  bool ok = true;
  for (int64_t k = nblk - 1; k > b; --k) {  // tile column b is full (b < k)
    const int64_t k0 = k * kBig;
    float4 lv[16];
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      const int64_t row = k0 + 16 * w + rr;
      lv[rr] = row < m ? __ldg(reinterpret_cast<const float4*>(L + row * ldm + r0 + 4 * lane))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    ok = warp_wait(flags, k, sc);
    if (!ok) break;
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      const int64_t row = k0 + 16 * w + rr;
      const float yv = row < m ? (float)__ldcg(y + row) : 0.f;
      colp[0] = fmaf(lv[rr].x, yv, colp[0]);
      colp[1] = fmaf(lv[rr].y, yv, colp[1]);
      colp[2] = fmaf(lv[rr].z, yv, colp[2]);
      colp[3] = fmaf(lv[rr].w, yv, colp[3]);
    }
  }
  *reinterpret_cast<float4*>(&sm.red[w][4 * lane]) = make_float4(colp[0], colp[1], colp[2], colp[3]);
  if (__syncthreads_or(!ok)) return;  // a wait gave up: the status says why
  if (tid < kBig) {
    float s = 0.f;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) s += sm.red[ww][tid];
    sm.rhs[tid] = tid < rb ? (float)zin[r0 + tid] - s : 0.f;
  }
  __syncthreads();
  const int r = tid & 127, h = tid >> 7;  // y_r = sum_c U_rc rhs_c, columns split in two halves
  float s = 0.f;
#pragma unroll 8
  for (int c = 64 * h; c < 64 * h + 64; ++c) s = fmaf(sm.U[r][c], sm.rhs[c], s);
  __syncthreads();  // (red is reused)
  sm.red[h][r] = s;
  __syncthreads();
  if (tid < rb) y[r0 + tid] = (double)(sm.red[0][tid] + sm.red[1][tid]);
  __threadfence();
  __syncthreads();
  if (tid == 0) st_release(flags + b, 1);
}

cudaError_t trsv_blk_prepare() {
  static bool done = false;  // per process; the attribute is per function
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_trsv_lower_blk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(TrsvSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_trsv_upper_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrsvSmem));
  if (e == cudaSuccess) done = true;
  return e;
}

}  // namespace

cudaError_t trsv_lower_blk(cudaStream_t st, int64_t m, int64_t ldm, const float* L, const float* Uinv,
                           const double* v, double* z, int* flags, unsigned* ticket, Scalars* sc) {
  const int64_t nblk = (m + kBig - 1) / kBig;
  cudaError_t e = trsv_blk_prepare();
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(int) * nblk, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  k_trsv_lower_blk<<<(unsigned)nblk, kThreads, sizeof(TrsvSmem), st>>>(m, ldm, L, Uinv, v, z, flags, ticket, sc);
  return cudaGetLastError();
}

cudaError_t trsv_upper_blk(cudaStream_t st, int64_t m, int64_t ldm, const float* L, const float* Uinv,
                           const double* z, double* y, int* flags, unsigned* ticket, Scalars* sc) {
  const int64_t nblk = (m + kBig - 1) / kBig;
  cudaError_t e = trsv_blk_prepare();
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(int) * nblk, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  k_trsv_upper_blk<<<(unsigned)nblk, kThreads, sizeof(TrsvSmem), st>>>(m, ldm, L, Uinv, z, y, flags, ticket, sc);
  return cudaGetLastError();
}

}  // namespace pdas
