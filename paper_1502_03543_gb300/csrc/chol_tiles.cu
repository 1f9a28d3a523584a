// chol_tiles.cu -- the Cholesky factor M = L L' of the normal matrix (the
// symmetric positive definite solve of Section V-A) as ONE persistent
// dataflow launch over 128 x 128 tiles, for the FP32 factor of the mixed
// forms.
//
// With 128-row tile indices i >= l and k < l, the tasks are
//   FINAL(l, l)    apply M_ll -= L_l,l-1 L_l,l-1', then L_ll = chol(M_ll)
//   FINAL(i, l)    apply M_il -= L_i,l-1 L_l,l-1', wait for FINAL(l, l),
//                  then L_il = M_il L_ll^{-T}
//   UPDATE(i,l,k)  M_il -= L_ik L_lk'   for k <= l - 2 (rank 128)
// A tile's last update and its factorisation or triangular solve run in one
// task on the tile held in registers, so the dependency chain of the
// factorisation (FINAL(l,l) -> FINAL(l+1,l) -> FINAL(l+1,l+1) ...) has no
// store, reload or hand-off between them.  Every tile (i, l) of the lower
// triangle has a counter in global memory: the number of updates applied to
// it, then l + 1 once it holds its final L values.
//
// CTAs take tasks from a ticket counter in a fixed list order.  In that order
// every task comes after all tasks it waits for, so a CTA only waits on tasks
// that running CTAs hold, and those finish by induction on the order; every
// wait is also bounded (2 s, PDAS_ERR_TIMEOUT).  The order itself comes from
// a list schedule simulated on the host for the number of resident CTAs:
// the ready task with the longest remaining path to the end of the
// factorisation (its "bottom level", from per-task cost estimates) goes
// first, which keeps the critical chain moving and fills the GPU with
// trailing updates around it.  A non-positive pivot records PDAS_ERR_NOT_SPD
// and its index; the other CTAs see the status and stop.
#include <algorithm>
#include <queue>
#include <vector>

#include "sync_util.cuh"
#include "tile_core.cuh"

namespace pdas {

namespace {

enum TileTask { TK_FINAL_DIAG = 0, TK_FINAL_OFF = 1, TK_UPDATE = 2, TK_INV = 3 };

// UPDATE operands: K chunks of 32 columns of two 128-row tile columns,
// row-major with a pitch of 36 floats / 34 doubles (16-byte rows, and 16
// consecutive rows fall in distinct 16-byte bank groups), double-buffered.
constexpr int kUpdK = 32;
template <typename T>
constexpr int upd_pitch() {
  return sizeof(T) == 4 ? 36 : 34;
}
template <typename T>
constexpr int upd_vec() {  // elements per 16-byte load
  return 16 / (int)sizeof(T);
}

template <typename T>
struct TileCholSmem {
  union {
    T stage[2][2][kBig][upd_pitch<T>()];  // UPDATE: [buffer][row tile i | row tile l][row][k]
    T ls[kBig][kBig + 1];                 // TRSM: the factor of the diagonal tile
  };
  T cb[2][kBig];  // column buffers of the POTRF / TRSM sweeps (double-buffered)
  T rcp[kBig];    // TRSM: 1 / L_cc; POTRF: the diagonal on entry
  int4 task;
  int go;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;  // 0: fill the 16 bytes with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T>
__device__ __forceinline__ bool pivot_bad(T d) {
  return !(d > T(0)) || !isfinite(d);
}

// Thread (tx, ty) holds rows ty + 16 i and columns tx + 16 j of a tile.  On a
// diagonal tile only the lower triangle is read and written.
template <typename T>
__device__ __forceinline__ void load_tile(T (&acc)[8][8], const T* M, int64_t ldm, int64_t m, int64_t p0, int64_t q0,
                                          bool diag) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t p = p0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t q = q0 + tx + 16 * j;
      acc[i][j] = (p < m && q < m && (!diag || q <= p)) ? __ldcg(M + p * ldm + q) : T(0);
    }
  }
}

template <typename T>
__device__ __forceinline__ void store_tile(const T (&acc)[8][8], T* M, int64_t ldm, int64_t m, int64_t p0,
                                           int64_t q0, bool diag) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t p = p0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t q = q0 + tx + 16 * j;
      if (p < m && q < m && (!diag || q <= p)) M[p * ldm + q] = acc[i][j];
    }
  }
}

// acc -= L_ik L_lk' for the tile (i, l) held in acc: four K chunks of 32
// columns, each copied into shared memory by asynchronous 16-byte copies (L2
// only) while the previous chunk is multiplied.  A step of the product reads
// 16 bytes along k for each of the thread's 8 rows, then, per column j, 16
// bytes of row j and 8 x VEC fused multiply-adds.  On a diagonal tile the
// thread's blocks j > i lie wholly above the diagonal and are skipped.  Tile
// column k is never the ragged last one (k < l), so every copied column is
// inside the matrix; rows past m are zero-filled.
template <typename T, bool DIAG>
__device__ __forceinline__ void rank_update(T (&acc)[8][8], int64_t m, int64_t ldm, const T* M, int i, int l, int k,
                                            TileCholSmem<T>& sm) {
  constexpr int VEC = upd_vec<T>();
  constexpr int CPR = kUpdK / VEC;  // 16-byte copies per row and chunk
  struct alignas(16) V {
    T v[VEC];
  };
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t p0 = (int64_t)i * kBig, q0 = (int64_t)l * kBig, k0 = (int64_t)k * kBig;
  auto issue = [&](int chunk, int buf) {
    const int64_t c0 = k0 + (int64_t)chunk * kUpdK;
#pragma unroll
    for (int e = tid; e < kBig * CPR; e += kThreads) {
      const int r = e / CPR, c = (e % CPR) * VEC;
      const bool pin = p0 + r < m;
      cp_async16(&sm.stage[buf][0][r][c], M + (pin ? (p0 + r) * ldm + c0 + c : 0), pin);
      if (!DIAG) {
        const bool qin = q0 + r < m;
        cp_async16(&sm.stage[buf][1][r][c], M + (qin ? (q0 + r) * ldm + c0 + c : 0), qin);
      }
    }
    cp_async_commit();
  };
  issue(0, 0);
  issue(1, 1);
  constexpr int NCH = kBig / kUpdK;
#pragma unroll 1
  for (int ch = 0; ch < NCH; ++ch) {
    const int buf = ch & 1;
    if (ch + 1 < NCH) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();
    const T(*P)[upd_pitch<T>()] = sm.stage[buf][0];
    const T(*Q)[upd_pitch<T>()] = sm.stage[buf][DIAG ? 0 : 1];
#pragma unroll 1
    for (int kk = 0; kk < kUpdK; kk += VEC) {
      V a[8];
#pragma unroll
      for (int ii = 0; ii < 8; ++ii) a[ii] = *reinterpret_cast<const V*>(&P[ty + 16 * ii][kk]);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const V b = *reinterpret_cast<const V*>(&Q[tx + 16 * j][kk]);
#pragma unroll
        for (int v = 0; v < VEC; ++v)
#pragma unroll
          for (int ii = 0; ii < 8; ++ii)
            if (!DIAG || j <= ii) acc[ii][j] = fma(-a[ii].v[v], b.v[v], acc[ii][j]);
      }
    }
    __syncthreads();
    if (ch + 2 < NCH) issue(ch + 2, buf);
  }
}

// 1 / sqrt(d): the hardware estimate refined by one Newton step (within
// about 2 ulp in FP32; the FP32 factor is a preconditioner); IEEE for FP64.
__device__ __forceinline__ float inv_sqrt(float d) {
  const float r = rsqrtf(d);
  return r * fmaf(-0.5f * d * r, r, 1.5f);
}
__device__ __forceinline__ double inv_sqrt(double d) { return 1.0 / sqrt(d); }

// Step C of the right-looking factorisation of a 32 x 32 block held by one
// warp (lane = row): the pivot comes by shuffle from lane C; every lane
// scales its entry of column C and publishes it in a 32-entry column buffer
// (double-buffered, so one warp barrier per step); each lane then reads the
// column entries it needs with 16-byte broadcast loads and updates its row.
// Recursion on C keeps every register index a compile-time constant.
template <typename T, int C>
__device__ __forceinline__ void warp_potrf_step(T (&row)[32], int lane, int& bad, T& myrs, T* cbuf) {
  const T d = __shfl_sync(0xffffffffu, row[C], C);
  if (bad < 0 && pivot_bad(d)) bad = C;  // (the sweep runs on; the block is discarded)
  const T rs = inv_sqrt(d);
  const T v = lane > C ? row[C] * rs : (lane == C ? d * rs : T(0));
  if (lane >= C) row[C] = v;
  if (lane == C) myrs = rs;
  T* col = cbuf + (C & 1) * 32;
  col[lane] = v;
  __syncwarp();
  constexpr int Q0 = (C + 1) & ~3;  // first 4-aligned group holding an entry q > C
#pragma unroll
  for (int q4 = Q0; q4 < 32; q4 += 4) {
    T c4[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) c4[e] = col[q4 + e];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int q = q4 + e;
      if (q > C && lane >= q) row[q] = fma(-v, c4[e], row[q]);
    }
  }
  if constexpr (C + 1 < 32) warp_potrf_step<T, C + 1>(row, lane, bad, myrs, cbuf);
}

// Factorisation of the diagonal tile (held in acc) through shared memory in
// four 32-column blocks; per block:
//   1. one warp factors the 32 x 32 diagonal block in registers (lane = row;
//      the pivot and the column entries it needs come by warp shuffles);
//   2. one thread per later row of the tile solves that row against it;
//   3. every thread updates the trailing lower triangle of the tile.
// Three block barriers per 32 columns.  Rows and columns past m (a ragged
// last tile) carry an identity diagonal, so they factor trivially and are not
// stored.  Returns false (status set) on a pivot that is not positive and
// finite.
template <typename T>
__device__ __forceinline__ bool tile_potrf(const T (&acc)[8][8], int64_t m, int64_t ldm, T* M, T* dinv, int l,
                                           TileCholSmem<T>& sm, Scalars* sc) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31, warp = tid >> 5;
  const int64_t p0 = (int64_t)l * kBig;
  const int kb = (int)(m - p0 < kBig ? m - p0 : kBig);
  T(*S)[kBig + 1] = sm.ls;
  __shared__ int s_fail;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = ty + 16 * i, q = tx + 16 * j;
      S[r][q] = (r >= kb && r == q) ? T(1) : acc[i][j];
    }
  if (tid == 0) s_fail = -1;
  __syncthreads();
  for (int b = 0; b < 4; ++b) {
    const int c0 = 32 * b;
    if (warp == 0) {  // 1. the diagonal block
      T row[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) row[q] = S[c0 + lane][c0 + q];
      int bad = -1;
      T myrs = T(1);
      warp_potrf_step<T, 0>(row, lane, bad, myrs, &sm.cb[0][0]);
      sm.rcp[c0 + lane] = myrs;
      if (bad >= 0) {
        if (lane == 0) s_fail = c0 + bad;
      } else {
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (q <= lane) S[c0 + lane][c0 + q] = row[q];
      }
    }
    __syncthreads();
    if (s_fail >= 0) break;
    const int r0 = c0 + 32, nr = kBig - r0;
    if (tid < nr) {  // 2. rows below: x L_bb' = s
      const int r = r0 + tid;
      T x[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) x[q] = S[r][c0 + q];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        x[c] *= sm.rcp[c0 + c];
#pragma unroll
        for (int q = c + 1; q < 32; ++q) x[q] = fma(-x[c], S[c0 + q][c0 + c], x[q]);
      }
#pragma unroll
      for (int q = 0; q < 32; ++q) S[r][c0 + q] = x[q];
    }
    __syncthreads();
    if (nr > 0) {  // 3. trailing lower triangle: S_rq -= sum_c S_r,c0+c S_q,c0+c
      const int nb16 = nr / 16;
      for (int i2 = 0; i2 < nb16; ++i2) {
        const int r = r0 + ty + 16 * i2;
        T a[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) a[c] = S[r][c0 + c];
        for (int j2 = 0; j2 <= i2; ++j2) {
          const int q = r0 + tx + 16 * j2;
          if (q <= r) {
            T v = S[r][q];
#pragma unroll
            for (int c = 0; c < 32; ++c) v = fma(-a[c], S[q][c0 + c], v);
            S[r][q] = v;
          }
        }
      }
    }
    __syncthreads();
  }
  if (s_fail >= 0) {
    if (tid == 0 && atomicCAS(&sc->status, 0, (int)PDAS_ERR_NOT_SPD) == 0) sc->fail_index = (int)(p0 + s_fail);
    return false;
  }
  for (int e = tid; e < kBig * kBig; e += kThreads) {
    const int r = e >> 7, q = e & 127;
    if (r < kb && q <= r) M[(p0 + r) * ldm + p0 + q] = S[r][q];
  }
  if (tid < kb) dinv[p0 + tid] = sm.rcp[tid];
  return true;
}

// Loads L_ll (strictly lower part; rows and columns past m read as the
// identity) and its pivot reciprocals into shared memory.
template <typename T>
__device__ __forceinline__ void load_diag_factor(int64_t m, int64_t ldm, const T* M, const T* dinv, int l,
                                                 TileCholSmem<T>& sm) {
  const int tid = threadIdx.x;
  const int64_t q0 = (int64_t)l * kBig;
  const int kb = (int)(m - q0 < kBig ? m - q0 : kBig);
  for (int e = tid; e < kBig * kBig; e += kThreads) {
    const int r = e >> 7, c = e & 127;
    sm.ls[r][c] = (c < r && r < kb) ? __ldcg(M + (q0 + r) * ldm + q0 + c) : T(0);
  }
  if (tid < kBig) sm.rcp[tid] = tid < kb ? __ldcg(dinv + q0 + tid) : T(1);
  __syncthreads();
}

// X L_ll' = C for the 128 rows held in acc, column by column with the pivot
// reciprocals (L_ll and 1 / L_cc in shared memory).  Row ty + 16 i of the
// tile lives in one half-warp (its 16 threads hold columns tx + 16 j), so the
// finished entry x = c_c / L_cc reaches the rest of its row by a width-16
// shuffle and the sweep needs no block barrier; every thread then subtracts
// x L_col,c from its later columns.
template <typename T>
__device__ __forceinline__ void trsm_sweep(T (&acc)[8][8], TileCholSmem<T>& sm) {
  const int tid = threadIdx.x, tx = tid & 15, half = tid & 16;
#pragma unroll
  for (int jo = 0; jo < 8; ++jo) {
#pragma unroll 1
    for (int cl = 0; cl < 16; ++cl) {
      const int c = 16 * jo + cl;
      const T rc = sm.rcp[c];
      T x[8];
#pragma unroll
      for (int ii = 0; ii < 8; ++ii) x[ii] = __shfl_sync(0xffffffffu, acc[ii][jo] * rc, half | cl);
      if (tx == cl) {
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) acc[ii][jo] = x[ii];
      }
#pragma unroll
      for (int j = jo; j < 8; ++j) {
        const int col = tx + 16 * j;
        const T bv = col > c ? sm.ls[col][c] : T(0);
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) acc[ii][j] = fma(-x[ii], bv, acc[ii][j]);
      }
    }
  }
}

// U_l = L_ll^{-T} (upper triangular; the identity past m): the sweep above
// applied to C = I.  Stored row-major 128 x 128 at Uinv + l 128^2; the
// blocked triangular solves apply it in place of a substitution.
template <typename T>
__device__ __forceinline__ void tile_inverse(T (&acc)[8][8], int64_t m, int64_t ldm, const T* M, const T* dinv,
                                             T* Uinv, int l, TileCholSmem<T>& sm) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  load_diag_factor<T>(m, ldm, M, dinv, l, sm);
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = (ty + 16 * i == tx + 16 * j) ? T(1) : T(0);
  trsm_sweep<T>(acc, sm);
  T* U = Uinv + (int64_t)l * kBig * kBig;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) U[(ty + 16 * i) * kBig + tx + 16 * j] = acc[i][j];
}

template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 2 : 1)
    k_chol_tiles(int64_t m, int64_t ldm, T* M, T* dinv, T* Uinv, const int4* __restrict__ tasks, int ntasks, int nb,
                 int* state, unsigned* ticket, Scalars* sc) {
  extern __shared__ __align__(16) unsigned char chol_tiles_smem[];
  TileCholSmem<T>& sm = *reinterpret_cast<TileCholSmem<T>*>(chol_tiles_smem);
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {  // take a task and wait for the tiles it starts from
      int go = 0;
      const unsigned t = atomicAdd(ticket, 1u);
      if (t < (unsigned)ntasks && !dev_failed(sc)) {
        const int4 d = tasks[t];
        sm.task = d;
        const int64_t i = d.y, l = d.z, k = d.w;
        if (d.x == TK_UPDATE)
          go = wait_at_least(state + i * nb + k, (int)k + 1, sc) && wait_at_least(state + l * nb + k, (int)k + 1, sc) &&
               wait_at_least(state + i * nb + l, (int)k, sc);
        else if (d.x == TK_INV)
          go = wait_at_least(state + l * nb + l, (int)l + 1, sc);
        else if (l == 0)
          go = 1;
        else
          go = wait_at_least(state + i * nb + l - 1, (int)l, sc) && wait_at_least(state + l * nb + l - 1, (int)l, sc) &&
               wait_at_least(state + i * nb + l, (int)l - 1, sc);
      }
      sm.go = go;
    }
    __syncthreads();
    if (!sm.go) return;
    const int4 d = sm.task;
    const int i = d.y, l = d.z;
    const int64_t p0 = (int64_t)i * kBig, q0 = (int64_t)l * kBig;
    T acc[8][8];
    int val;
    if (d.x == TK_INV) {
      tile_inverse<T>(acc, m, ldm, M, dinv, Uinv, l, sm);
      __syncthreads();  // (shared memory is reused by the next task; no counter to publish)
      continue;
    }
    if (d.x == TK_UPDATE) {
      load_tile(acc, M, ldm, m, p0, q0, i == l);
      if (i == l) rank_update<T, true>(acc, m, ldm, M, i, l, d.w, sm);
      else rank_update<T, false>(acc, m, ldm, M, i, l, d.w, sm);
      store_tile(acc, M, ldm, m, p0, q0, i == l);
      val = d.w + 1;
    } else if (d.x == TK_FINAL_DIAG) {
      load_tile(acc, M, ldm, m, p0, p0, true);
      if (l > 0) rank_update<T, true>(acc, m, ldm, M, l, l, l - 1, sm);
      if (!tile_potrf<T>(acc, m, ldm, M, dinv, l, sm, sc)) return;
      val = l + 1;
    } else {
      load_tile(acc, M, ldm, m, p0, q0, false);
      if (l > 0) rank_update<T, false>(acc, m, ldm, M, i, l, l - 1, sm);
      if (tid == 0) sm.go = wait_at_least(state + (int64_t)l * nb + l, l + 1, sc);  // L_ll
      __syncthreads();
      if (!sm.go) return;
      load_diag_factor<T>(m, ldm, M, dinv, l, sm);
      trsm_sweep<T>(acc, sm);
      store_tile(acc, M, ldm, m, p0, q0, false);
      val = l + 1;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release(state + (int64_t)i * nb + l, val);
  }
}

}  // namespace

template <typename T>
size_t chol_tiles_smem_bytes() {
  return sizeof(TileCholSmem<T>);
}

int64_t chol_tile_count(int64_t m) { return (m + kBig - 1) / kBig; }

// Resident CTAs of the FP32 tile Cholesky on the current device (the worker
// count the task order is scheduled for).
int chol_tiles_resident() {
  cudaError_t e = cudaFuncSetAttribute(k_chol_tiles<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)chol_tiles_smem_bytes<float>());
  int occ = 0, dev = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_chol_tiles<float>, kThreads,
                                                      chol_tiles_smem_bytes<float>());
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || occ < 1 || sms < 1) {
    cudaGetLastError();
    return 0;
  }
  return occ * sms;
}

// The task order (see the file comment): a list schedule of the task graph
// on nproc identical workers.  Costs are relative estimates per task kind
// (a diagonal update skips about 44% of the products; the triangular solve
// and the factorisation sweep 128 columns with a block barrier each).
void chol_tile_tasks(int64_t m, int nproc, std::vector<int4>* out) {
  const int nb = (int)chol_tile_count(m);
  out->clear();
  if (nb <= 0 || nb > kTileCholMaxTiles) return;
  if (nproc < 1) nproc = 1;
  constexpr double kUpd = 31.0, kUpdDiag = 18.0, kPotrf = 63.0, kTrsm = 46.0, kInv = 46.0;
  struct Node {
    int4 d;
    double pre, post;  // cost before / after the mid-task wait (FINAL(i, l): for L_ll)
    int mid;           // FINAL(l, l) for FINAL(i, l), i > l; else -1
    int npred;
  };
  std::vector<Node> nodes;
  std::vector<std::vector<int>> succ;
  // index maps: FINAL(i, l) -> fidx[i nb + l]; UPDATE(i, l, k) -> ubase[l nb + k] + i - l
  std::vector<int> fidx((size_t)nb * nb, -1), ubase((size_t)nb * nb, -1);
  auto add = [&](int4 d, double pre, double post) {
    nodes.push_back(Node{d, pre, post, -1, 0});
    return (int)nodes.size() - 1;
  };
  for (int l = 0; l < nb; ++l) {
    fidx[(size_t)l * nb + l] = add(make_int4(TK_FINAL_DIAG, l, l, l - 1), (l ? kUpdDiag : 0.0) + kPotrf, 0.0);
    add(make_int4(TK_INV, l, l, 0), kInv, 0.0);
    for (int i = l + 1; i < nb; ++i) fidx[(size_t)i * nb + l] = add(make_int4(TK_FINAL_OFF, i, l, l - 1), l ? kUpd : 0.0, kTrsm);
    for (int k = 0; k + 2 <= l; ++k) {
      ubase[(size_t)l * nb + k] = (int)nodes.size();
      for (int i = l; i < nb; ++i) add(make_int4(TK_UPDATE, i, l, k), i == l ? kUpdDiag : kUpd, 0.0);
    }
  }
  succ.resize(nodes.size());
  auto edge = [&](int a, int b) {
    succ[a].push_back(b);
    ++nodes[b].npred;
  };
  auto upd = [&](int i, int l, int k) { return ubase[(size_t)l * nb + k] + (i - l); };
  for (int v = 0; v < (int)nodes.size(); ++v) {
    const int4 d = nodes[v].d;
    const int i = d.y, l = d.z, k = d.w;
    if (d.x == TK_INV) {
      edge(fidx[(size_t)l * nb + l], v);
    } else if (d.x == TK_UPDATE) {
      edge(fidx[(size_t)i * nb + k], v);
      if (l != i) edge(fidx[(size_t)l * nb + k], v);
      if (k > 0) edge(upd(i, l, k - 1), v);
    } else {
      if (l > 0) {
        edge(fidx[(size_t)i * nb + l - 1], v);
        if (i != l) edge(fidx[(size_t)l * nb + l - 1], v);
        if (l >= 2) edge(upd(i, l, l - 2), v);
      }
      if (d.x == TK_FINAL_OFF) nodes[v].mid = fidx[(size_t)l * nb + l];
    }
  }
  // bottom levels (nodes were created in a topological order of the start
  // edges; the mid edge FINAL(l,l) -> FINAL(i,l) also goes forward)
  const int N = (int)nodes.size();
  std::vector<double> bl(N, 0.0);
  std::vector<std::vector<int>> midsucc(N);
  for (int v = 0; v < N; ++v)
    if (nodes[v].mid >= 0) midsucc[nodes[v].mid].push_back(v);
  for (int v = N - 1; v >= 0; --v) {
    double best = 0.0;
    for (int w : succ[v]) best = std::max(best, bl[w]);
    for (int w : midsucc[v]) best = std::max(best, bl[w]);
    bl[v] = nodes[v].pre + nodes[v].post + best;
  }
  // list schedule
  std::vector<char> handed(N, 0), startable(N, 0);
  std::vector<double> fin(N, 0.0);
  auto cmp = [&](int a, int b) { return bl[a] < bl[b] || (bl[a] == bl[b] && a > b); };
  std::priority_queue<int, std::vector<int>, decltype(cmp)> ready(cmp);
  auto try_ready = [&](int v) {
    if (startable[v] && !handed[v] && (nodes[v].mid < 0 || handed[nodes[v].mid])) {
      handed[v] = 2;  // queued
      ready.push(v);
    }
  };
  for (int v = 0; v < N; ++v)
    if (nodes[v].npred == 0) {
      startable[v] = 1;
      try_ready(v);
    }
  using Ev = std::pair<double, int>;  // finish time, node
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> running;
  double t = 0.0;
  int busy = 0;
  out->reserve(N);
  while ((int)out->size() < N) {
    while (busy < nproc && !ready.empty()) {
      const int v = ready.top();
      ready.pop();
      handed[v] = 1;
      out->push_back(nodes[v].d);
      double f = t + nodes[v].pre;
      if (nodes[v].mid >= 0) f = std::max(f, fin[nodes[v].mid]);
      f += nodes[v].post;
      fin[v] = f;
      running.push(Ev(f, v));
      ++busy;
      for (int w : midsucc[v]) try_ready(w);
    }
    if (running.empty()) break;  // (cannot happen: the graph is acyclic)
    const Ev e = running.top();
    running.pop();
    t = e.first;
    --busy;
    for (int w : succ[e.second])
      if (--nodes[w].npred == 0) {
        startable[w] = 1;
        try_ready(w);
      }
  }
}

template <typename T>
cudaError_t cholesky_tiles(cudaStream_t st, int64_t m, int64_t ldm, T* M, T* dinv, T* Uinv, const int4* tasks,
                           int ntasks, int* state, unsigned* ticket, Scalars* sc) {
  static int per_sm = 0;  // resident CTAs per SM (per process; the attribute is per function)
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_chol_tiles<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)chol_tiles_smem_bytes<T>());
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_chol_tiles<T>, kThreads, chol_tiles_smem_bytes<T>());
    if (e != cudaSuccess) return e;
    per_sm = occ > 0 ? occ : 1;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int nb = (int)chol_tile_count(m);
  e = cudaMemsetAsync(state, 0, sizeof(int) * (size_t)nb * nb, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  int grid = sms * per_sm;
  if (grid > ntasks) grid = ntasks;
  k_chol_tiles<T><<<grid, kThreads, chol_tiles_smem_bytes<T>(), st>>>(m, ldm, M, dinv, Uinv, tasks, ntasks, nb,
                                                                     state, ticket, sc);
  return cudaGetLastError();
}

template cudaError_t cholesky_tiles<float>(cudaStream_t, int64_t, int64_t, float*, float*, float*, const int4*, int,
                                           int*, unsigned*, Scalars*);
template cudaError_t cholesky_tiles<double>(cudaStream_t, int64_t, int64_t, double*, double*, double*, const int4*,
                                            int, int*, unsigned*, Scalars*);

}  // namespace pdas

// Host-only: the task order, for tests of its dependency structure.
extern "C" int64_t pdas_chol_tile_tasks(int64_t m, int32_t nproc, int32_t* out, int64_t cap) {
  if (m <= 0) return 0;
  std::vector<int4> t;
  pdas::chol_tile_tasks(m, nproc, &t);
  const int64_t n = (int64_t)t.size();
  if (out) {
    for (int64_t e = 0; e < n && e < cap; ++e) {
      out[4 * e] = t[e].x;
      out[4 * e + 1] = t[e].y;
      out[4 * e + 2] = t[e].z;
      out[4 * e + 3] = t[e].w;
    }
  }
  return n;
}
