// chol.cu -- blocked right-looking Cholesky M = L L' of the normal matrix and
// the two triangular solves L z = r, L' dy = z: the symmetric positive
// definite solve of (A D A') dy = A x (Section V-A names Cholesky as the
// usual route; here it is blocked so the O(m^3) work is a rank-64 update).
//
// Per 64-column panel k0:
//   k_chol_panel  -- every block factors the 64 x 64 diagonal block in shared
//                    memory; block 0 writes it back, blocks >= 1 each solve 64
//                    panel rows X L11' = B with four threads per row;
//   k_chol_update -- trailing lower tiles C -= P P' (the SIMT tile core).
// A pivot that is not positive (or not finite) sets PDAS_ERR_NOT_SPD with its
// index in the device status; later launches see the status and do nothing.
//
// The triangular solves are one launch each.  Blocks take row blocks in
// order from a ticket counter; block b waits (bounded, ~2 s) for the flags of
// the blocks it depends on, so a block only waits on blocks that were handed
// out earlier and are running or done -- no deadlock.  On a timeout it sets
// PDAS_ERR_TIMEOUT and returns.
#include "sync_util.cuh"
#include "tile_core.cuh"

namespace pdas {

namespace {

template <typename T>
__device__ __forceinline__ bool pivot_bad(T d) {
  return !(d > T(0)) || !isfinite(d);
}

// 1 / sqrt(d) of a pivot, or -1 for a pivot that is not positive and finite.
template <typename T>
__device__ __forceinline__ T pivot_rp(T d) {
  return pivot_bad(d) ? T(-1) : T(1) / sqrt(d);
}

// Factor the kb x kb diagonal block held in shared memory (lower triangle).
// Right-looking by columns with two barriers per column: column c is scaled
// by rp_c = 1 / sqrt(d_c), d_c = Ld[c][c] (no thread writes the diagonal
// during the loop; it is replaced by sqrt(d_c) at the end), then the trailing
// block is updated.  Thread (ti, tj) = (tid / 16, tid % 16) updates rows
// ti + 16 k and columns tj + 16 l.  rp_c is computed once, by thread 0, as
// soon as d_c is final (thread 0 updates entry (c, c) first in the update of
// column c - 1) and passed on in shared memory: on GPUs whose FP64 pipes run
// at a small fraction of the FP32 rate, a square root and a division in
// every thread would cost more than the whole update.
// Returns -1 or the local index of the failing pivot (same in all threads).
template <typename T>
__device__ int factor_diag(T (*Ld)[kTile + 1], int kb) {
  __shared__ T s_rp[2];
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
  if (threadIdx.x == 0 && kb > 0) s_rp[0] = pivot_rp(Ld[0][0]);
  for (int c = 0; c < kb; ++c) {
    __syncthreads();  // the trailing update of column c - 1 is complete, rp_c posted
    const T rp = s_rp[c & 1];
    if (rp < T(0)) return c;
    for (int r = c + 1 + threadIdx.x; r < kb; r += blockDim.x) Ld[r][c] *= rp;
    __syncthreads();  // column c is scaled
    for (int i = c + 1 + ti; i < kb; i += 16) {
      const T lic = Ld[i][c];
      for (int j = c + 1 + tj; j <= i; j += 16) {
        Ld[i][j] -= lic * Ld[j][c];
        if (i == c + 1 && j == c + 1) s_rp[(c + 1) & 1] = pivot_rp(Ld[i][j]);  // thread 0: d_c+1 is final
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < kb) Ld[threadIdx.x][threadIdx.x] = sqrt(Ld[threadIdx.x][threadIdx.x]);
  __syncthreads();
  return -1;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_chol_panel(int64_t m, int64_t ldm, T* M, T* dinv, int64_t k0, int kb,
                                                         Scalars* sc) {
  __shared__ T Ld[kTile][kTile + 1];
  __shared__ T rcp[kTile];  // 1 / L_cc: the row solves multiply (GB300's FP64 division is a long sequence)
  if (dev_failed(sc)) return;
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, j = e % kb;
    Ld[i][j] = j <= i ? M[(k0 + i) * ldm + k0 + j] : T(0);
  }
  __syncthreads();
  const int fail = factor_diag<T>(Ld, kb);
  if (fail >= 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && atomicCAS(&sc->status, 0, (int)PDAS_ERR_NOT_SPD) == 0)
      sc->fail_index = (int)(k0 + fail);
    return;
  }
  if (threadIdx.x < kb) rcp[threadIdx.x] = T(1) / Ld[threadIdx.x][threadIdx.x];
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
      const int i = e / kb, j = e % kb;
      if (j <= i) M[(k0 + i) * ldm + k0 + j] = Ld[i][j];
    }
    if (threadIdx.x < kb) dinv[k0 + threadIdx.x] = rcp[threadIdx.x];
    return;
  }
  // Panel rows: X L11' = B, right-looking over columns; thread (row, part)
  // owns columns part, part+4, ... of its row in registers.
  const int row = threadIdx.x >> 2, part = threadIdx.x & 3;
  const int64_t i = k0 + kb + (int64_t)(blockIdx.x - 1) * kTile + row;
  const bool live = i < m;
  T b[kTile / 4];
#pragma unroll
  for (int k = 0; k < kTile / 4; ++k) {
    const int c = part + 4 * k;
    b[k] = (live && c < kb) ? M[i * ldm + k0 + c] : T(0);
  }
#pragma unroll
  for (int c = 0; c < kTile; ++c) {
    if (c < kb) {
      const int owner = c & 3;
      T xc = (part == owner) ? b[c >> 2] * rcp[c] : T(0);
      xc = __shfl_sync(0xffffffffu, xc, (threadIdx.x & 31 & ~3) | owner);
      if (part == owner) b[c >> 2] = xc;
#pragma unroll
      for (int k = 0; k < kTile / 4; ++k) {
        const int cp = part + 4 * k;
        if (cp > c && cp < kb) b[k] -= xc * Ld[cp][c];
      }
    }
  }
  if (live) {
#pragma unroll
    for (int k = 0; k < kTile / 4; ++k) {
      const int c = part + 4 * k;
      if (c < kb) M[i * ldm + k0 + c] = b[k];
    }
  }
}

// Trailing update C -= P P' over 128 x 128 lower tiles of the trailing matrix
// (P = the kb <= 64 panel columns).  Every load is issued up front -- the C
// tile straight into the accumulators, both 128 x kb panels into shared
// memory (transposed, so the products read broadcasts and consecutive
// words) -- then the kb rank-1 steps run from shared memory.  Thread
// (tx, ty) owns rows ty + 16 i and columns tx + 16 j of the tile.
template <typename T>
constexpr size_t update_smem_bytes() {
  return 2 * sizeof(T) * kTile * (kBig + 1);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 2 : 1) k_chol_update(int64_t m, int64_t ldm, T* M, int64_t k0, int kb,
                                                          const Scalars* sc) {
  extern __shared__ __align__(16) unsigned char update_smem[];
  T(*Ps)[kBig + 1] = reinterpret_cast<T(*)[kBig + 1]>(update_smem);
  T(*Qs)[kBig + 1] = reinterpret_cast<T(*)[kBig + 1]>(update_smem + sizeof(T) * kTile * (kBig + 1));
  if (dev_failed(sc)) return;
  int64_t ti, tj;
  lower_tile(blockIdx.x, ti, tj);
  const int64_t s0 = k0 + kb;
  const int64_t p0 = s0 + ti * kBig, q0 = s0 + tj * kBig;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t p = p0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t q = q0 + tx + 16 * j;
      acc[i][j] = (p < m && q <= p) ? M[p * ldm + q] : T(0);
    }
  }
#pragma unroll 4
  for (int e = threadIdx.x; e < kBig * kTile; e += kThreads) {
    const int r = e / kTile, c = e % kTile;  // a warp reads 32 consecutive panel columns of one row
    const bool cin = c < kb;
    Ps[c][r] = (cin && p0 + r < m) ? M[(p0 + r) * ldm + k0 + c] : T(0);
    Qs[c][r] = (cin && q0 + r < m) ? M[(q0 + r) * ldm + k0 + c] : T(0);
  }
  __syncthreads();
  for (int c = 0; c < kb; ++c) {
    T a[8], b[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = Ps[c][ty + 16 * i];
#pragma unroll
    for (int j = 0; j < 8; ++j) b[j] = Qs[c][tx + 16 * j];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fma(-a[i], b[j], acc[i][j]);
  }
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

// Reduce-scatter of eight per-lane partial sums v[0..7] over the warp: every
// lane returns the whole sum of row red_row(lane) = 4 b4 + 2 b3 + b2 (b_k bit
// k of the lane), with 9 additions (5 levels) where summing the eight rows
// one by one takes 40: on GPUs whose FP64 pipes are charged per warp
// instruction the difference is ~2000 cycles per block.
template <typename T>
__device__ __forceinline__ T warp_reduce_scatter8(const T (&v)[8], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
  T a[4], b[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {  // lanes 0-15 keep rows 0-3, lanes 16-31 rows 4-7
    const T keep = h16 ? v[i + 4] : v[i], give = h16 ? v[i] : v[i + 4];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const T keep = h8 ? a[i + 2] : a[i], give = h8 ? a[i] : a[i + 2];
    b[i] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
  }
  T c = (h4 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, h4 ? b[0] : b[1], 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}
__device__ __forceinline__ int red_row(int lane) { return 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1); }

// ---------------------------------------------------------------------------
// L z = v.  Block row b (64 rows): z_b = L_bb^{-1} (v_b - sum_{j<b} L_bj z_j).
// Arithmetic in T (the factor's precision; the FP32 factor of the mixed forms
// is a preconditioner, refined in FP64 afterwards); v, z in FP64.  Warp w
// owns rows 8w..8w+7 of the block, lane l owns columns l, l+32; the diagonal
// block is solved by warp 0.  SCALED (the FP64 tier of the mixed forms,
// whose refinement takes the solve as a preconditioner): on its rows divided
// by their pivots, z_r = v_r / L_rr - sum_{c<r} (L_rc / L_rr) z_c, so a step
// of its chain is one shuffle and one multiply-add, and the eight row sums
// of a warp are combined by a reduce-scatter.  Otherwise (the plain FP64
// form's direct solve, Section V-A) by substitution with the pivot
// reciprocals and a butterfly per row.
template <typename T, bool SCALED>
__global__ void __launch_bounds__(kThreads) k_trsv_lower(int64_t m, int64_t ldm, const T* __restrict__ L,
                                                         const T* __restrict__ dinv, const double* __restrict__ v,
                                                         double* z, int* flags, unsigned* ticket, Scalars* sc) {
  __shared__ T Ld[kTile][kTile + 1];
  __shared__ T acc[kTile];
  __shared__ T rcp[kTile];
  __shared__ int sbi;
  if (threadIdx.x == 0) sbi = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  if (dev_failed(sc)) return;
  const int64_t b = sbi;
  const int64_t r0 = b * kTile;
  const int rb = (int)(m - r0 < kTile ? m - r0 : kTile);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int i = e / kTile, j = e % kTile;
    Ld[i][j] = (i < rb && j < i) ? L[(r0 + i) * ldm + r0 + j] * (SCALED ? dinv[r0 + i] : T(1)) : T(0);  // row i over L_ii
  }
  if (threadIdx.x < kTile) rcp[threadIdx.x] = threadIdx.x < rb ? dinv[r0 + threadIdx.x] : T(0);
  T part[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) part[i] = T(0);
  bool ok = true;
  for (int64_t jb = 0; jb < b && ok; ++jb) {
    T l0[8], l1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = 8 * w + i;
      const T* row = L + (r0 + r) * ldm + jb * kTile;
      l0[i] = r < rb ? row[lane] : T(0);
      l1[i] = r < rb ? row[lane + 32] : T(0);
    }
    ok = warp_wait(flags, jb, sc);
    if (!ok) break;
    // lane l needs exactly z_{jb*64 + l} and z_{jb*64 + l + 32}
    const T z0 = (T)__ldcg(z + jb * kTile + lane);
    const T z1 = (T)__ldcg(z + jb * kTile + lane + 32);
#pragma unroll
    for (int i = 0; i < 8; ++i) part[i] = fma(l0[i], z0, fma(l1[i], z1, part[i]));
  }
  if constexpr (SCALED) {
    const T t = warp_reduce_scatter8(part, lane);
    const int r = 8 * w + red_row(lane);
    if ((lane & 3) == 0) acc[r] = r < rb ? (T)v[r0 + r] - t : T(0);
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      T t = part[i];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      const int r = 8 * w + i;
      if (lane == 0) acc[r] = r < rb ? (T)v[r0 + r] - t : T(0);
    }
  }
  if (__syncthreads_or(!ok)) return;  // a wait gave up: the status says why
  if (w == 0) {
    T a0, a1;
    if constexpr (SCALED) {
      // the scaled right-hand side; rows 0..31 finish at column 31, so the
      // second half of the sweep updates a1 only
      a0 = acc[lane] * rcp[lane];
      a1 = acc[lane + 32] * rcp[lane + 32];
      const int c1 = rb < 32 ? rb : 32;
      for (int c = 0; c < c1; ++c) {
        const T zc = __shfl_sync(0xffffffffu, a0, c);
        if (lane > c) a0 = fma(-Ld[lane][c], zc, a0);
        a1 = fma(-Ld[lane + 32][c], zc, a1);
      }
      for (int c = 32; c < rb; ++c) {
        const T zc = __shfl_sync(0xffffffffu, a1, c - 32);
        if (lane + 32 > c) a1 = fma(-Ld[lane + 32][c], zc, a1);
      }
    } else {
      a0 = acc[lane];
      a1 = acc[lane + 32];
      for (int c = 0; c < rb; ++c) {
        const T own = c < 32 ? a0 : a1;
        const T zc = __shfl_sync(0xffffffffu, own, c & 31) * rcp[c];
        if (lane == (c & 31)) {
          if (c < 32) a0 = zc;
          else a1 = zc;
        }
        if (lane > c) a0 -= Ld[lane][c] * zc;
        if (lane + 32 > c) a1 -= Ld[lane + 32][c] * zc;
      }
    }
    if (lane < rb) z[r0 + lane] = (double)a0;
    if (lane + 32 < rb) z[r0 + lane + 32] = (double)a1;
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(flags + b, 1);
  }
}

// L' y = z.  Row block b of L' is column block b of L; blocks go from the
// last to the first.  For each later block kb, thread (w, lane) adds
// L[k][r] y_k for rows k = 8w..8w+7 of that block and columns r = lane, lane+32.
template <typename T, bool SCALED>
__global__ void __launch_bounds__(kThreads) k_trsv_upper_t(int64_t m, int64_t ldm, const T* __restrict__ L,
                                                           const T* __restrict__ dinv,
                                                           const double* __restrict__ zin, double* y, int* flags,
                                                           unsigned* ticket, Scalars* sc) {
  __shared__ T Ld[kTile][kTile + 1];
  __shared__ T red[8][kTile];
  __shared__ T rcp[kTile];
  __shared__ int sbi;
  const int64_t nblk = (m + kTile - 1) / kTile;
  if (threadIdx.x == 0) sbi = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  if (dev_failed(sc)) return;
  const int64_t b = nblk - 1 - sbi;
  const int64_t r0 = b * kTile;
  const int rb = (int)(m - r0 < kTile ? m - r0 : kTile);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int i = e / kTile, j = e % kTile;
    Ld[i][j] = (i < rb && j < i) ? L[(r0 + i) * ldm + r0 + j] * (SCALED ? dinv[r0 + j] : T(1)) : T(0);  // column j over L_jj
  }
  if (threadIdx.x < kTile) rcp[threadIdx.x] = threadIdx.x < rb ? dinv[r0 + threadIdx.x] : T(0);
  T p0 = T(0), p1 = T(0);
  bool ok = true;
  for (int64_t kb = nblk - 1; kb > b && ok; --kb) {
    const int64_t k0 = kb * kTile;
    const int kr = (int)(m - k0 < kTile ? m - k0 : kTile);
    T l0[8], l1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = 8 * w + i;
      const T* row = L + (k0 + k) * ldm + r0;
      l0[i] = (k < kr && lane < rb) ? row[lane] : T(0);
      l1[i] = (k < kr && lane + 32 < rb) ? row[lane + 32] : T(0);
    }
    ok = warp_wait(flags, kb, sc);
    if (!ok) break;
    // warp w needs y_{k0 + 8w .. k0 + 8w + 7}: the same values in every lane
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = 8 * w + i;
      const T yv = k < kr ? (T)__ldcg(y + k0 + k) : T(0);
      p0 = fma(l0[i], yv, p0);
      p1 = fma(l1[i], yv, p1);
    }
  }
  red[w][lane] = p0;
  red[w][lane + 32] = p1;
  if (__syncthreads_or(!ok)) return;  // a wait gave up: the status says why
  if (w == 0) {
    T a0 = T(0), a1 = T(0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      a0 += red[i][lane];
      a1 += red[i][lane + 32];
    }
    a0 = lane < rb ? (T)zin[r0 + lane] - a0 : T(0);
    a1 = lane + 32 < rb ? (T)zin[r0 + lane + 32] - a1 : T(0);
    if constexpr (SCALED) {
      // rows divided by their pivots (the coefficients were scaled at the
      // load): a step of the chain is one shuffle and one multiply-add
      a0 *= rcp[lane];
      a1 *= rcp[lane + 32];
      for (int c = rb - 1; c >= 32; --c) {
        const T yc = __shfl_sync(0xffffffffu, a1, c - 32);
        if (lane + 32 < c) a1 = fma(-Ld[c][lane + 32], yc, a1);
        a0 = fma(-Ld[c][lane], yc, a0);
      }
      for (int c = (rb < 32 ? rb : 32) - 1; c >= 0; --c) {
        const T yc = __shfl_sync(0xffffffffu, a0, c);
        if (lane < c) a0 = fma(-Ld[c][lane], yc, a0);
      }
    } else {
      for (int c = rb - 1; c >= 0; --c) {
        const T own = c < 32 ? a0 : a1;
        const T yc = __shfl_sync(0xffffffffu, own, c & 31) * rcp[c];
        if (lane == (c & 31)) {
          if (c < 32) a0 = yc;
          else a1 = yc;
        }
        if (lane < c) a0 -= Ld[c][lane] * yc;
        if (lane + 32 < c) a1 -= Ld[c][lane + 32] * yc;
      }
    }
    if (lane < rb) y[r0 + lane] = (double)a0;
    if (lane + 32 < rb) y[r0 + lane + 32] = (double)a1;
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(flags + b, 1);
  }
}

}  // namespace

template <typename T>
cudaError_t cholesky(cudaStream_t st, int64_t m, int64_t ldm, T* M, T* dinv, Scalars* sc) {
  static bool attr_set = false;  // per process; the attribute is per function
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_chol_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)update_smem_bytes<T>());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  for (int64_t k0 = 0; k0 < m; k0 += kTile) {
    const int kb = (int)(m - k0 < kTile ? m - k0 : kTile);
    const int64_t rest = m - k0 - kb;
    const int64_t t = (rest + kTile - 1) / kTile;
    const int64_t tu = (rest + kBig - 1) / kBig;
    k_chol_panel<T><<<(unsigned)(1 + t), kThreads, 0, st>>>(m, ldm, M, dinv, k0, kb, sc);
    if (tu > 0)
      k_chol_update<T><<<(unsigned)(tu * (tu + 1) / 2), kThreads, update_smem_bytes<T>(), st>>>(m, ldm, M, k0, kb,
                                                                                              sc);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t trsv_lower(cudaStream_t st, int64_t m, int64_t ldm, const T* L, const T* dinv, const double* v, double* z,
                       int* flags, unsigned* tickets, Scalars* sc, bool scaled) {
  const int64_t nblk = (m + kTile - 1) / kTile;
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int) * nblk, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(tickets + T_TRSV, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (scaled)
    k_trsv_lower<T, true><<<(unsigned)nblk, kThreads, 0, st>>>(m, ldm, L, dinv, v, z, flags, tickets + T_TRSV, sc);
  else
    k_trsv_lower<T, false><<<(unsigned)nblk, kThreads, 0, st>>>(m, ldm, L, dinv, v, z, flags, tickets + T_TRSV, sc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t trsv_upper_t(cudaStream_t st, int64_t m, int64_t ldm, const T* L, const T* dinv, const double* z,
                         double* y, int* flags, unsigned* tickets, Scalars* sc, bool scaled) {
  const int64_t nblk = (m + kTile - 1) / kTile;
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int) * nblk, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(tickets + T_TRSV, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (scaled)
    k_trsv_upper_t<T, true><<<(unsigned)nblk, kThreads, 0, st>>>(m, ldm, L, dinv, z, y, flags, tickets + T_TRSV, sc);
  else
    k_trsv_upper_t<T, false><<<(unsigned)nblk, kThreads, 0, st>>>(m, ldm, L, dinv, z, y, flags, tickets + T_TRSV, sc);
  return cudaGetLastError();
}

template cudaError_t cholesky<double>(cudaStream_t, int64_t, int64_t, double*, double*, Scalars*);
template cudaError_t cholesky<float>(cudaStream_t, int64_t, int64_t, float*, float*, Scalars*);
template cudaError_t trsv_lower<double>(cudaStream_t, int64_t, int64_t, const double*, const double*, const double*,
                                        double*, int*, unsigned*, Scalars*, bool);
template cudaError_t trsv_lower<float>(cudaStream_t, int64_t, int64_t, const float*, const float*, const double*,
                                       double*, int*, unsigned*, Scalars*, bool);
template cudaError_t trsv_upper_t<double>(cudaStream_t, int64_t, int64_t, const double*, const double*, const double*,
                                          double*, int*, unsigned*, Scalars*, bool);
template cudaError_t trsv_upper_t<float>(cudaStream_t, int64_t, int64_t, const float*, const float*, const double*,
                                         double*, int*, unsigned*, Scalars*, bool);

}  // namespace pdas
