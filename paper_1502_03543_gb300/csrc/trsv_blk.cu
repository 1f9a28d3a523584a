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
// counter and wait (bounded: 2 s, or the handle's own limit) for the
// solution blocks they depend on, which were handed out earlier: no
// deadlock.  The solution vector is filled
// with an all-ones bit pattern before the launch (a value the solves cannot
// produce: each entry is an FP32 sum widened to FP64, whose low 29 bits are
// zero), and a consumer polls the entries it needs until none holds it, so
// the hand-off from block to block is one round trip to L2, with no flag and
// no fence.  Thread layout for the off-diagonal tiles: warp w holds rows
// 16 w .. 16 w + 15, lane l columns 4 l .. 4 l + 3 (16-byte loads along the
// rows); tiles are loaded before the wait for the block they multiply.
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

constexpr unsigned long long kUnset = ~0ull;  // the fill of a solution entry not yet written

__device__ __forceinline__ double ld_relaxed_f64(const double* p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_f64(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// The warp waits (bounded) until none of the N entries p[k * stride] (k < N,
// this lane's share) holds kUnset; entries with valid[k] false are not
// waited for and read as 0.  Returns false on a timeout or a failed status.
template <int N>
__device__ __forceinline__ bool poll_entries(const double* p, const bool (&valid)[N], double (&out)[N], Scalars* sc) {
  const uint64_t t0 = global_ns(), limit = wait_limit_ns(sc);
  for (;;) {
    bool mine = true;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      out[k] = valid[k] ? ld_relaxed_f64(p + k) : 0.0;
      mine = mine && __double_as_longlong(out[k]) != (long long)kUnset;
    }
    if (__all_sync(0xffffffffu, mine)) return true;
    if (dev_failed(sc)) return false;
    if (global_ns() - t0 > limit) {
      atomicCAS(&sc->status, 0, (int)PDAS_ERR_TIMEOUT);
      return false;
    }
    __nanosleep(32);
  }
}

__device__ __forceinline__ void load_u(TrsvSmem& sm, const float* __restrict__ Ub) {
  for (int e = threadIdx.x; e < kBig * kBig; e += blockDim.x) sm.U[e >> 7][e & 127] = __ldg(Ub + e);
}

// L z = v: z_b = U_b' (v_b - sum_{j<b} L_bj z_j).
__global__ void __launch_bounds__(kThreads, 1) k_trsv_lower_blk(int64_t m, int64_t ldm, const float* __restrict__ L,
                                                             const float* __restrict__ Uinv,
                                                             const double* __restrict__ v, double* z,
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
  const int myrow = 16 * w + ((lane >> 1) & 15);  // the row this lane finishes after the reduction
  const float vmine = myrow < rb ? (float)v[r0 + myrow] : 0.f;  // off the dependency chain
  float part[16];
#pragma unroll
  for (int rr = 0; rr < 16; ++rr) part[rr] = 0.f;
  bool ok = true;
  // Two buffers: block j + 1's tile rows and solution entries are in flight
  // while block j's products run (entries read too early are re-polled).
  float4 lv[2][16];
  double zd[2][4];
  auto fetch = [&](int64_t j, int buf) {  // tile j is full (j < b <= nb - 1)
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      const int64_t row = r0 + 16 * w + rr;
      lv[buf][rr] = row < m ? __ldg(reinterpret_cast<const float4*>(L + row * ldm + j * kBig + 4 * lane))
                            : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) zd[buf][k] = ld_relaxed_f64(z + j * kBig + 4 * lane + k);
  };
  auto consume = [&](int64_t j, int buf) {
    bool mine = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) mine = mine && __double_as_longlong(zd[buf][k]) != (long long)kUnset;
    if (!__all_sync(0xffffffffu, mine)) {
      const bool all4[4] = {true, true, true, true};
      if (!poll_entries<4>(z + j * kBig + 4 * lane, all4, zd[buf], sc)) return false;
    }
    const float z0 = (float)zd[buf][0], z1 = (float)zd[buf][1], z2 = (float)zd[buf][2], z3 = (float)zd[buf][3];
#pragma unroll
    for (int rr = 0; rr < 16; ++rr)
      part[rr] = fmaf(lv[buf][rr].x, z0, fmaf(lv[buf][rr].y, z1, fmaf(lv[buf][rr].z, z2, fmaf(lv[buf][rr].w, z3, part[rr]))));
    return true;
  };
  if (b > 0) fetch(0, 0);
  for (int64_t j = 0; j < b && ok; j += 2) {
    if (j + 1 < b) fetch(j + 1, 1);
    ok = consume(j, 0);
    if (!ok || j + 1 >= b) break;
    if (j + 2 < b) fetch(j + 2, 0);
    ok = consume(j + 1, 1);
  }
  const float tot = reduce16(part, lane);
  if ((lane & 1) == 0) sm.rhs[myrow] = myrow < rb ? vmine - tot : 0.f;
  if (__syncthreads_or(!ok)) return;  // a wait gave up: the status says why
  const int c = tid & 127, h = tid >> 7;  // z_c = sum_r U_rc rhs_r, rows split in two halves
  float s = 0.f;
#pragma unroll 8
  for (int r = 64 * h; r < 64 * h + 64; ++r) s = fmaf(sm.U[r][c], sm.rhs[r], s);
  sm.red[h][c] = s;
  __syncthreads();
  if (tid < rb) st_relaxed_f64(z + r0 + tid, (double)(sm.red[0][tid] + sm.red[1][tid]));
}

// L' y = z: y_b = U_b (z_b - sum_{k>b} L_kb' y_k); blocks go from the last.
__global__ void __launch_bounds__(kThreads, 1) k_trsv_upper_blk(int64_t m, int64_t ldm, const float* __restrict__ L,
                                                             const float* __restrict__ Uinv,
                                                             const double* __restrict__ zin, double* y,
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
  const float zmine = tid < rb ? (float)zin[r0 + tid] : 0.f;  // off the dependency chain
  float colp[4] = {0.f, 0.f, 0.f, 0.f};  // columns 4 lane .. 4 lane + 3 of tile b, this warp's rows
  bool ok = true;
  // Two buffers, as in the forward solve: block k - 1's tile rows and
  // solution entries are in flight while block k's products run.  Lane l
  // holds entry 16 w + (l & 15) of a block of y; the warp shares them.
  float4 lv[2][16];
  double yd[2];
  auto fetch = [&](int64_t k, int buf) {  // tile column b is full (b < k)
    const int64_t k0 = k * kBig;
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      const int64_t row = k0 + 16 * w + rr;
      lv[buf][rr] = row < m ? __ldg(reinterpret_cast<const float4*>(L + row * ldm + r0 + 4 * lane))
                            : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int64_t mine = k0 + 16 * w + (lane & 15);
    yd[buf] = mine < m ? ld_relaxed_f64(y + mine) : 0.0;
  };
  auto consume = [&](int64_t k, int buf) {
    const int64_t k0 = k * kBig, mine = k0 + 16 * w + (lane & 15);
    if (!__all_sync(0xffffffffu, __double_as_longlong(yd[buf]) != (long long)kUnset)) {
      const bool inside[1] = {mine < m};
      double one[1];
      if (!poll_entries<1>(y + mine, inside, one, sc)) return false;
      yd[buf] = one[0];
    }
    const float ymine = (float)yd[buf];
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      const float yv = __shfl_sync(0xffffffffu, ymine, rr);
      colp[0] = fmaf(lv[buf][rr].x, yv, colp[0]);
      colp[1] = fmaf(lv[buf][rr].y, yv, colp[1]);
      colp[2] = fmaf(lv[buf][rr].z, yv, colp[2]);
      colp[3] = fmaf(lv[buf][rr].w, yv, colp[3]);
    }
    return true;
  };
  if (nblk - 1 > b) fetch(nblk - 1, 0);
  for (int64_t k = nblk - 1; k > b && ok; k -= 2) {
    if (k - 1 > b) fetch(k - 1, 1);
    ok = consume(k, 0);
    if (!ok || k - 1 <= b) break;
    if (k - 2 > b) fetch(k - 2, 0);
    ok = consume(k - 1, 1);
  }
  *reinterpret_cast<float4*>(&sm.red[w][4 * lane]) = make_float4(colp[0], colp[1], colp[2], colp[3]);
  if (__syncthreads_or(!ok)) return;  // a wait gave up: the status says why
  if (tid < kBig) {
    float s = 0.f;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) s += sm.red[ww][tid];
    sm.rhs[tid] = tid < rb ? zmine - s : 0.f;
  }
  __syncthreads();
  const int r = tid & 127, h = tid >> 7;  // y_r = sum_c U_rc rhs_c, columns split in two halves
  float s = 0.f;
#pragma unroll 8
  for (int c = 64 * h; c < 64 * h + 64; ++c) s = fmaf(sm.U[r][c], sm.rhs[c], s);
  __syncthreads();  // (red is reused)
  sm.red[h][r] = s;
  __syncthreads();
  if (tid < rb) st_relaxed_f64(y + r0 + tid, (double)(sm.red[0][tid] + sm.red[1][tid]));
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
                           const double* v, double* z, unsigned* ticket, Scalars* sc) {
  const int64_t nblk = (m + kBig - 1) / kBig;
  cudaError_t e = trsv_blk_prepare();
  if (e == cudaSuccess) e = cudaMemsetAsync(z, 0xff, sizeof(double) * m, st);  // every entry kUnset
  if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  k_trsv_lower_blk<<<(unsigned)nblk, kThreads, sizeof(TrsvSmem), st>>>(m, ldm, L, Uinv, v, z, ticket, sc);
  return cudaGetLastError();
}

cudaError_t trsv_upper_blk(cudaStream_t st, int64_t m, int64_t ldm, const float* L, const float* Uinv,
                           const double* z, double* y, unsigned* ticket, Scalars* sc) {
  const int64_t nblk = (m + kBig - 1) / kBig;
  cudaError_t e = trsv_blk_prepare();
  if (e == cudaSuccess) e = cudaMemsetAsync(y, 0xff, sizeof(double) * m, st);  // every entry kUnset
  if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  k_trsv_upper_blk<<<(unsigned)nblk, kThreads, sizeof(TrsvSmem), st>>>(m, ldm, L, Uinv, z, y, ticket, sc);
  return cudaGetLastError();
}

}  // namespace pdas
