// chol_tiles.cu -- the Cholesky factor M = L L' of the normal matrix (the
// symmetric positive definite solve of Section V-A) as ONE persistent
// dataflow launch over 128 x 128 tiles, for the FP32 factor of the mixed
// forms.
//
// With 128-row tile indices i >= l and k < l, the tasks are
//   FINAL(l, l)    apply M_ll -= L_l,l-1 L_l,l-1', then L_ll = chol(M_ll)
//   FINAL(i, l)    apply M_il -= L_i,l-1 L_l,l-1', wait for FINAL(l, l),
//                  then L_il = M_il L_ll^{-T}   (i >= l + 2)
//   SOLVE(l+1, l)  L_l+1,l = M_l+1,l L_ll^{-T}  (all its updates applied)
//   UPDATE(i,l,k)  M_il -= L_ik L_lk'   for k <= l - 2, and for k = l - 1
//                  when i = l + 1 (rank 128)
// In the FP32 factor every product L_ik L_lk' runs on the tcgen05 tensor
// cores (BF16 operand planes, FP32 accumulation in tensor memory; see the
// section "FP32 products on the tensor cores"); the FP64 instantiation keeps
// SIMT products.
// A tile's last update and its factorisation or triangular solve run in one
// task on the tile held in registers (except the sub-diagonal tiles, see
// below), and the dependency chain of the factorisation (FINAL(l,l) ->
// SOLVE(l+1,l) -> FINAL(l+1,l+1) ...) runs in one CTA.  Every tile (i, l) of
// the lower triangle has a counter in global memory: the number of updates
// applied to it, then l + 1 once it holds its final L values.
//
// Block 0 runs the dependency chain itself: FINAL(l, l), then the solve of
// the sub-diagonal tile (l + 1, l) against L_ll while L_ll and its pivot
// reciprocals are still in its shared memory (that tile's last update,
// k = l - 1, is an ordinary UPDATE task), then FINAL(l + 1, l + 1), ...  The
// head of the chain never queues behind trailing updates, and no chain link
// crosses between CTAs.  The
// other CTAs take the remaining tasks from a ticket counter in a fixed list
// order.  In that order every task comes after all tasks it waits for (block
// 0's tasks included), so the first unfinished task is always held by a
// running CTA and has all it waits for done, and every task finishes by
// induction on the order; every wait is also bounded (2 s, PDAS_ERR_TIMEOUT).
// The order itself comes from
// a list schedule simulated on the host for the number of resident CTAs:
// the ready task with the longest remaining path to the end of the
// factorisation (its "bottom level", from per-task cost estimates) goes
// first, which keeps the critical chain moving and fills the GPU with
// trailing updates around it.  A non-positive pivot records PDAS_ERR_NOT_SPD
// and its index; the other CTAs see the status and stop.
#include <algorithm>
#include <type_traits>
#include <queue>
#include <vector>

#include <cuda_bf16.h>

#include "sync_util.cuh"
#include "tc_util.cuh"
#include "df_util.cuh"
#include "tile_core.cuh"

namespace pdas {

namespace {

enum TileTask { TK_FINAL_DIAG = 0, TK_FINAL_OFF = 1, TK_UPDATE = 2, TK_INV = 3, TK_CHAIN_SOLVE = 4 };

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

// Tensor-core products (FP32 factor).  Every finished off-diagonal tile of L
// is stored once more as three BF16 planes (x = x0 + x1 + x2, 8 significant
// bits apiece, so every product of planes is exact in FP32), per K chunk of
// 64 columns: 128 rows x 128 bytes with the 128-byte swizzle, the layout the
// MMA reads from shared memory.  A product copies the chunks of both operand
// tiles into shared memory with bulk copies (the tensor memory accelerator)
// and multiplies them there.
constexpr int kTcPlaneBytes = kBig * 128;          // one plane of one K chunk
constexpr int kTcChunkBytes = 3 * kTcPlaneBytes;   // the three planes of one operand's K chunk
constexpr int kTcTileBytes = 2 * kTcChunkBytes;    // one tile: both K chunks (its slot in the plane buffer)
constexpr int kTcBufBytes = 2 * kTcChunkBytes;     // one K chunk in shared memory: A planes | B planes
constexpr int kTcOpsBytes = 2 * kTcBufBytes;       // both K chunks
constexpr uint32_t kTcCols = 256;                  // TMEM: leading term | the five correction terms
constexpr uint32_t kTcIdesc = tc::idesc_bf16(kBig, kBig);

// Slot of the off-diagonal tile (i, k), i > k, in the plane buffer.
__host__ __device__ constexpr int64_t plane_slot(int64_t i, int64_t k) { return i * (i - 1) / 2 + k; }

template <typename T>
struct TileCholSmem {
  union {
    T stage[2][2][kBig][upd_pitch<T>()];  // UPDATE (FP64): [buffer][row tile i | row tile l][row][k]
    T ls[kBig][kBig + 1];                 // TRSM: the factor of the diagonal tile; FP32 products: D
    unsigned char tc_ops[kTcOpsBytes + 1024];  // FP32 products: the BF16 planes (1024-aligned inside)
  };
  T cb[2][kBig];  // column buffers of the POTRF / TRSM sweeps (double-buffered)
  T rcp[kBig];    // TRSM: 1 / L_cc; POTRF: the diagonal on entry
  unsigned long long mma_bar;      // FP32 products: completion of the issued MMAs
  unsigned long long full_bar[2];  // FP32 products: arrival of the K chunks' planes
  uint32_t tmem_slot;
  int tc_ok;
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

// One element from global memory through L2 (the tile counters order it after
// its producer's release).
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ dfloat ld_cg(const dfloat* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return dfloat(v.x, v.y);
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
      acc[i][j] = (p < m && q < m && (!diag || q <= p)) ? ld_cg(M + p * ldm + q) : T(0);
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

// 1 / sqrt(d) of a pivot: the hardware estimate (within 2 ulp in FP32; the
// FP32 factor is a preconditioner, and every entry of a column is scaled by
// the same value); IEEE for FP64.
__device__ __forceinline__ float inv_sqrt(float d) { return rsqrtf(d); }
__device__ __forceinline__ double inv_sqrt(double d) { return 1.0 / sqrt(d); }

// Right-looking factorisation of a 32 x 32 block held by one warp (lane =
// row), as a loop over the pivot column C: row[] is shifted left every step,
// so row[0] always holds column C and the loop body has fixed register
// indices.  Per step the lane of row C + 1 forms the next pivot from its own
// new entry and broadcasts it (one shuffle on the dependency chain); the new
// column goes to a 32-entry window of a shared buffer (indexed relative to
// C, double-buffered) that every lane reads with 16-byte loads to update its
// later entries.  Finished entries of column C go to out[C] (out = this
// lane's row of the block; rows above the diagonal are not written).
template <typename T>
__device__ __forceinline__ void warp_potrf(T (&row)[32], int lane, int& bad, T& myrs, T* cbuf, T* out) {
  constexpr int VN = 16 / (int)sizeof(T);
  struct alignas(16) V {
    T v[VN];
  };
  T d = __shfl_sync(0xffffffffu, row[0], 0);
#pragma unroll 1
  for (int C = 0; C < 32; ++C) {
    if (bad < 0 && pivot_bad(d)) bad = C;  // (the sweep runs on; the block is discarded)
    const T rs = inv_sqrt(d);
    const T v = lane > C ? row[0] * rs : (lane == C ? d * rs : T(0));
    if (lane >= C) out[C] = v;
    if (lane == C) myrs = rs;
    const T dn = __shfl_sync(0xffffffffu, fma(-v, v, row[1]), (C + 1) & 31);
    T* col = cbuf + (C & 1) * 64;
    col[lane - C + 32] = v;  // entry q (relative to C) at 32 + q; lanes below C write below the window
    __syncwarp();
#pragma unroll
    for (int q4 = 0; q4 < 32; q4 += VN) {
      const V c4 = *reinterpret_cast<const V*>(col + 32 + q4);
#pragma unroll
      for (int e = 0; e < VN; ++e)
        if (q4 + e >= 1) row[q4 + e] = fma(-v, c4.v[e], row[q4 + e]);
    }
#pragma unroll
    for (int q = 0; q < 31; ++q) row[q] = row[q + 1];
    d = dn;
  }
}

// S_rq -= sum_{c < 32} S_r,c0+c S_q,c0+c for the entries r >= rlo, qlo <= q < qhi
// of the tile in shared memory, in 4 x 4 units (those wholly above the
// diagonal skipped; entries above it inside a unit are updated and never
// read), spread over the P threads p = 0..P-1 of the caller.
template <typename T>
__device__ __forceinline__ void potrf_trail(T (*S)[kBig + 1], int c0, int rlo, int qlo, int qhi, int p, int P) {
  const int nq4 = (qhi - qlo) >> 2, nunits = ((kBig - rlo) >> 2) * nq4;
#pragma unroll 1
  for (int u = p; u < nunits; u += P) {
    const int r = rlo + 4 * (u / nq4), q = qlo + 4 * (u % nq4);
    if (q > r + 3) continue;
    T t[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) t[i][j] = S[r + i][q + j];
#pragma unroll 4
    for (int c = 0; c < 32; ++c) {
      T a[4], bq[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = S[r + i][c0 + c];
        bq[i] = S[q + i][c0 + c];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) t[i][j] = fma(-a[i], bq[j], t[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) S[r + i][q + j] = t[i][j];
  }
}

// The finished panel c0 .. c0 + 31 (rows r >= c0 inside the matrix, lower
// part) to global memory, by the P threads p of the caller.
template <typename T>
__device__ __forceinline__ void potrf_store_panel(const T (*S)[kBig + 1], T* M, int64_t ldm, int64_t p0, int kb, int c0,
                                                  int p, int P) {
#pragma unroll 4
  for (int e = p; e < (kBig - c0) * 32; e += P) {
    const int r = c0 + (e >> 5), c = c0 + (e & 31);
    if (r < kb && c <= r) M[(p0 + r) * ldm + p0 + c] = S[r][c];
  }
}

// Factorisation of the diagonal tile (held in acc) through shared memory in
// four 32-column blocks, right-looking with a look-ahead of one block.  Per
// block b (columns c0 = 32 b ..):
//   1. warp 0 factors the 32 x 32 diagonal block (warp_potrf); meanwhile the
//      other warps apply block b - 1 to the columns past this block and
//      store block b - 1;
//   2. one thread per later row solves that row against the block;
//   3. every thread applies block b to the next block's columns only.
// Three block barriers per block.  Rows and columns past m (a ragged last
// tile) carry an identity diagonal, so they factor trivially and are not
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
#pragma unroll 1
  for (int b = 0; b < 4; ++b) {
    const int c0 = 32 * b;
    if (warp == 0) {  // 1. the diagonal block
      T row[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) row[q] = S[c0 + lane][c0 + q];
      int bad = -1;
      T myrs = T(1);
      warp_potrf<T>(row, lane, bad, myrs, &sm.cb[0][0], &S[c0 + lane][c0]);
      sm.rcp[c0 + lane] = myrs;
      if (bad >= 0 && lane == 0) s_fail = c0 + bad;
    } else if (b > 0) {  // 1'. block b - 1 on the columns past block b, and its store
      potrf_trail<T>(S, c0 - 32, c0 + 32, c0 + 32, kBig, tid - 32, kThreads - 32);
      potrf_store_panel<T>(S, M, ldm, p0, kb, c0 - 32, tid - 32, kThreads - 32);
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
    if (nr > 0) {  // 3. the next block's columns
      potrf_trail<T>(S, c0, r0, r0, r0 + 32, tid, kThreads);
      __syncthreads();
    }
  }
  if (s_fail >= 0) {
    if (tid == 0 && atomicCAS(&sc->status, 0, (int)PDAS_ERR_NOT_SPD) == 0) sc->fail_index = (int)(p0 + s_fail);
    return false;
  }
  potrf_store_panel<T>(S, M, ldm, p0, kb, 96, tid, kThreads);
  if (tid < kb) dinv[p0 + tid] = sm.rcp[tid];
  return true;
}

// 16-byte vectors of T in registers (component access by constant index).
template <typename T>
struct Vec16Reg;
template <>
struct Vec16Reg<float> {
  using V = float4;
  static constexpr int N = 4;
  __device__ static V load(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
  __device__ static float get(const V& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
  __device__ static V make(const float (&a)[4]) { return make_float4(a[0], a[1], a[2], a[3]); }
};
template <>
struct Vec16Reg<dfloat> {
  using V = float4;
  static constexpr int N = 2;
  __device__ static V load(const dfloat* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
  __device__ static dfloat get(const V& v, int k) { return k == 0 ? dfloat(v.x, v.y) : dfloat(v.z, v.w); }
  __device__ static V make(const dfloat (&a)[2]) { return make_float4(a[0].hi, a[0].lo, a[1].hi, a[1].lo); }
};
template <>
struct Vec16Reg<double> {
  using V = double2;
  static constexpr int N = 2;
  __device__ static V load(const double* p) { return __ldcg(reinterpret_cast<const double2*>(p)); }
  __device__ static double get(const V& v, int k) { return k == 0 ? v.x : v.y; }
  __device__ static V make(const double (&a)[2]) { return make_double2(a[0], a[1]); }
};

// Loads L_ll (strictly lower part; rows and columns past m read as the
// identity) and its pivot reciprocals into shared memory: 16-byte loads,
// issued in batches of eight before their stores.
template <typename T>
__device__ __forceinline__ void load_diag_factor(int64_t m, int64_t ldm, const T* M, const T* dinv, int l,
                                                 TileCholSmem<T>& sm) {
  using R = Vec16Reg<T>;
  constexpr int VN = R::N;
  constexpr int VPR = kBig / VN;              // vectors per row
  constexpr int PER = kBig * VPR / kThreads;  // vectors per thread
  constexpr int BATCH = 8;                    // in flight per thread (the caller holds its tile in registers)
  static_assert(PER % BATCH == 0, "whole batches");
  const int tid = threadIdx.x;
  const int64_t q0 = (int64_t)l * kBig;
  const int kb = (int)(m - q0 < kBig ? m - q0 : kBig);
#pragma unroll 1
  for (int u0 = 0; u0 < PER; u0 += BATCH) {
    typename R::V buf[BATCH];
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const int e = tid + kThreads * (u0 + u), r = e / VPR, c = (e % VPR) * VN;
      const T* src = M + (q0 + r) * ldm + q0 + c;
      if (r < kb && c + VN <= r + 1) {  // every column of the vector is <= r < kb: inside the matrix
        buf[u] = R::load(src);
      } else {
        T a[VN];
#pragma unroll
        for (int k = 0; k < VN; ++k) a[k] = (c + k < r && r < kb) ? ld_cg(src + k) : T(0);
        buf[u] = R::make(a);
      }
    }
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const int e = tid + kThreads * (u0 + u), r = e / VPR, c = (e % VPR) * VN;
#pragma unroll
      for (int k = 0; k < VN; ++k) sm.ls[r][c + k] = c + k < r ? R::get(buf[u], k) : T(0);
    }
  }
  if (tid < kBig) sm.rcp[tid] = tid < kb ? ld_cg(dinv + q0 + tid) : T(1);
  __syncthreads();
}

// X L_ll' = C for the 128 rows held in acc, column by column with the pivot
// reciprocals (L_ll and 1 / L_cc in shared memory).  Row ty + 16 i of the
// tile lives in one half-warp (its 16 threads hold columns tx + 16 j): the
// thread of column c scales its 8 entries to x = c_c / L_cc and posts them in
// a per-half-warp slot of shared memory (two 16-byte stores; slots alternate
// with the column parity), and after a warp barrier the other threads of the
// half-warp read them (two 16-byte broadcast loads) and subtract x L_col,c
// from their later columns.  No block barrier in the sweep.
template <typename T>
__device__ __forceinline__ void trsm_sweep(T (&acc)[8][8], TileCholSmem<T>& sm) {
  constexpr int VN = 16 / (int)sizeof(T);
  struct alignas(16) V {
    T v[VN];
  };
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T* slots = &sm.cb[0][0];  // [column parity][half-warp ty][8 rows]
#pragma unroll
  for (int jo = 0; jo < 8; ++jo) {
#pragma unroll 1
    for (int cl = 0; cl < 16; ++cl) {
      const int c = 16 * jo + cl;
      T* slot = slots + ((c & 1) * 16 + ty) * 8;
      if (tx == cl) {
        const T rc = sm.rcp[c];
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) acc[ii][jo] *= rc;
#pragma unroll
        for (int v = 0; v < 8; v += VN) {
          V w;
#pragma unroll
          for (int e = 0; e < VN; ++e) w.v[e] = acc[v + e][jo];
          *reinterpret_cast<V*>(slot + v) = w;
        }
      }
      __syncwarp();
      T x[8];
#pragma unroll
      for (int v = 0; v < 8; v += VN) {
        const V w = *reinterpret_cast<const V*>(slot + v);
#pragma unroll
        for (int e = 0; e < VN; ++e) x[v + e] = w.v[e];
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
  __syncwarp();
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

// ---- FP32 products on the tensor cores ---------------------------------------
// D = L_ik L_lk' for one tile column k (K = 128) of the FP32 factor, with
// every operand split into three BF16 planes: the leading term A0 B0' goes
// to TMEM columns [0, 128), the five terms A0 B1' + A1 B0' + A0 B2' + A1 B1' +
// A2 B0' (each at most 2^-8 of it) to columns [128, 256).  The dropped terms
// are below 2^-24 relative, so the sum carries FP32 accuracy; the tensor
// core's FP32 accumulation rounds toward zero, and keeping the leading term
// in an accumulator of its own holds that to 8 accumulation steps.

// x = x0 + x1 + x2 with x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1)
// (each difference exact in FP32), for the pair (a, b): word s holds the
// BF16 term s of a (low half) and of b (high half).
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ void bf16x2_split3(float a, float b, uint32_t& w0, uint32_t& w1, uint32_t& w2) {
  w0 = bf16x2_bits(a, b);
  const float ra = a - __uint_as_float(w0 << 16), rb = b - __uint_as_float(w0 & 0xffff0000u);
  w1 = bf16x2_bits(ra, rb);
  const float sa = ra - __uint_as_float(w1 << 16), sb = rb - __uint_as_float(w1 & 0xffff0000u);
  w2 = bf16x2_bits(sa, sb);
}

constexpr int kStagePitch = kBig + 4;  // FP32 staging rows: 16-byte aligned; 8 consecutive rows in distinct bank groups
static_assert(kBig * kStagePitch * (int)sizeof(float) <= kTcOpsBytes, "the staging area lies inside the planes");

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// The BF16 planes of the finished tile held in acc (tile layout) to its slot
// of the plane buffer.  The tile passes through a staging area as FP32 rows;
// thread item e (8 per thread) is K chunk e / 1024, row (e / 8) % 128 and
// 16-byte chunk e % 8 of that row.  Rows past m hold zeros in acc.
__device__ __forceinline__ void tc_write_planes(const float (&acc)[8][8], unsigned char* slot, TileCholSmem<float>& sm) {
  float(*S)[kStagePitch] = reinterpret_cast<float(*)[kStagePitch]>(sm.tc_ops);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  __syncthreads();  // (the staging area overlaps L_ll)
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) S[ty + 16 * i][tx + 16 * j] = acc[i][j];
  __syncthreads();
#pragma unroll 2
  for (int u = 0; u < 2 * kBig * 8 / kThreads; ++u) {
    const int e = tid + kThreads * u, kc = e >> 10, r = (e >> 3) & (kBig - 1), c8 = e & 7;
    const float4 lo = *reinterpret_cast<const float4*>(&S[r][64 * kc + 8 * c8]);
    const float4 hi = *reinterpret_cast<const float4*>(&S[r][64 * kc + 8 * c8 + 4]);
    uint32_t w[3][4];
    bf16x2_split3(lo.x, lo.y, w[0][0], w[1][0], w[2][0]);
    bf16x2_split3(lo.z, lo.w, w[0][1], w[1][1], w[2][1]);
    bf16x2_split3(hi.x, hi.y, w[0][2], w[1][2], w[2][2]);
    bf16x2_split3(hi.z, hi.w, w[0][3], w[1][3], w[2][3]);
    unsigned char* dst = slot + kc * kTcChunkBytes + r * 128 + ((c8 ^ (r & 7)) << 4);
#pragma unroll
    for (int sp = 0; sp < 3; ++sp)
      *reinterpret_cast<uint4*>(dst + sp * kTcPlaneBytes) = make_uint4(w[sp][0], w[sp][1], w[sp][2], w[sp][3]);
  }
  asm volatile("fence.proxy.async.global;" ::: "memory");  // read next by bulk copies (async proxy)
}

// One thread: the 24 MMAs of a K chunk (A planes at ops, B planes after them
// or, on a diagonal tile, the A planes again).
__device__ __forceinline__ void tc_issue(uint32_t ops, bool diag, uint32_t tmem, bool first) {
  const uint32_t a0 = ops, a1 = ops + kTcPlaneBytes, a2 = ops + 2 * kTcPlaneBytes;
  const uint32_t b0 = diag ? ops : ops + kTcChunkBytes, b1 = b0 + kTcPlaneBytes, b2 = b0 + 2 * kTcPlaneBytes;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {  // K = 16 per MMA: 32 bytes along the swizzled row
    const uint32_t acc = (first && ks == 0) ? 0u : 1u;
    const uint64_t da0 = tc::sdesc_sw128(a0) + 2 * ks, da1 = tc::sdesc_sw128(a1) + 2 * ks,
                   da2 = tc::sdesc_sw128(a2) + 2 * ks;
    const uint64_t db0 = tc::sdesc_sw128(b0) + 2 * ks, db1 = tc::sdesc_sw128(b1) + 2 * ks,
                   db2 = tc::sdesc_sw128(b2) + 2 * ks;
    tc::umma_f16(tmem, da0, db0, kTcIdesc, acc);
    tc::umma_f16(tmem + kBig, da0, db1, kTcIdesc, acc);
    tc::umma_f16(tmem + kBig, da1, db0, kTcIdesc, 1u);
    tc::umma_f16(tmem + kBig, da0, db2, kTcIdesc, 1u);
    tc::umma_f16(tmem + kBig, da1, db1, kTcIdesc, 1u);
    tc::umma_f16(tmem + kBig, da2, db0, kTcIdesc, 1u);
  }
}

// D = L_ia L_ib' for the tiles in plane slots ta, tb (ta == tb on a diagonal
// tile).  Thread 0 copies both K chunks of both operands into shared memory
// and issues each chunk's MMAs once its planes have landed; the other threads
// go on (the caller overlaps its loads of C) and meet at tc_product_end.  Every
// barrier completes once per product, so one parity bit serves all three.
template <bool DIAG>
__device__ __forceinline__ void tc_product_begin(const unsigned char* planes, int64_t ta, int64_t tb,
                                                 TileCholSmem<float>& sm, uint32_t tmem, uint32_t parity,
                                                 Scalars* sc) {
  if (threadIdx.x != 0) return;
  unsigned char* ops = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sm.tc_ops) + 1023) & ~uintptr_t(1023));
  const uint32_t ops_s = tc::smem_u32(ops);
  asm volatile("fence.proxy.async.global;" ::: "memory");  // the planes were published by generic stores
  const unsigned char* A = planes + ta * kTcTileBytes;
  const unsigned char* B = planes + tb * kTcTileBytes;
#pragma unroll
  for (int kc = 0; kc < 2; ++kc) {
    const uint32_t bar = tc::smem_u32(&sm.full_bar[kc]);
    tc::mbar_expect_tx(bar, DIAG ? kTcChunkBytes : 2 * kTcChunkBytes);
    bulk_copy(ops_s + kc * kTcBufBytes, A + kc * kTcChunkBytes, kTcChunkBytes, bar);
    if (!DIAG) bulk_copy(ops_s + kc * kTcBufBytes + kTcChunkBytes, B + kc * kTcChunkBytes, kTcChunkBytes, bar);
  }
  int ok = 1;
#pragma unroll
  for (int kc = 0; kc < 2; ++kc) {
    if (ok && !tc::mbar_wait(tc::smem_u32(&sm.full_bar[kc]), parity, nullptr)) ok = 0;
    if (ok) {
      tc::fence_after();
      tc_issue(ops_s + kc * kTcBufBytes, DIAG, tmem, kc == 0);
    }
  }
  tc::umma_commit(tc::smem_u32(&sm.mma_bar));
  if (!ok) {  // a copy did not land in time: record it and let the copies drain (bounded)
    atomicCAS(&sc->status, 0, (int)PDAS_ERR_TIMEOUT);
    for (int kc = 0; kc < 2; ++kc) tc::mbar_wait(tc::smem_u32(&sm.full_bar[kc]), parity, nullptr);
  }
  sm.tc_ok = ok;
}

// Every thread: bounded wait for the product's MMAs; false (for all threads)
// on a timeout here or in tc_product_begin.
__device__ __forceinline__ bool tc_product_end(TileCholSmem<float>& sm, uint32_t& parity, Scalars* sc) {
  const uint32_t bar = tc::smem_u32(&sm.mma_bar);
  bool ok = tc::mbar_wait(bar, parity, nullptr);
  if (!ok) {
    atomicCAS(&sc->status, 0, (int)PDAS_ERR_TIMEOUT);
    tc::mbar_wait(bar, parity, nullptr);  // let the MMAs drain before TMEM is freed
  }
  parity ^= 1u;
  tc::fence_after();
  const int all = __syncthreads_and(ok);
  return all && sm.tc_ok;
}

// UPDATE epilogue: C -= D on the tile (p0, q0) in global memory, by whole
// rows with 16-byte accesses: warp w owns rows w + 8 j (j = 0..15), lane the
// columns 4 lane .. + 3.  tc_load_rows prefetches the warp's rows of C (while
// the last MMAs run); tc_sub_global drains TMEM (warp w: lanes 32 (w % 4) ..
// + 31, one row per thread, columns 64 (w / 4) .. + 63) into a staging area
// (the operand planes are free once the MMAs completed) and applies it.  On a
// diagonal tile only q <= p is written.
constexpr int kRowsPerWarp = kBig / (kThreads / 32);

__device__ __forceinline__ void tc_load_rows(float4 (&x)[kRowsPerWarp], int64_t m, int64_t ldm, const float* M,
                                             int64_t p0, int64_t q0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = q0 + 4 * lane;
#pragma unroll
  for (int j = 0; j < kRowsPerWarp; ++j) {
    const int64_t p = p0 + warp + (kThreads / 32) * j;
    x[j] = (p < m && q + 3 < m) ? __ldcg(reinterpret_cast<const float4*>(M + p * ldm + q)) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

template <bool DIAG>
__device__ __forceinline__ void tc_sub_global(float4 (&x)[kRowsPerWarp], int64_t m, int64_t ldm, float* M, int64_t p0,
                                              int64_t q0, uint32_t tmem, TileCholSmem<float>& sm) {
  float(*S)[kStagePitch] = reinterpret_cast<float(*)[kStagePitch]>(sm.tc_ops);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, quarter = warp & 3, half = warp >> 2;
  const int r = quarter * 32 + lane;
  const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
  for (int g = 0; g < 4; ++g) {
    const int c = half * 64 + g * 16;
    uint32_t lead[16], corr[16];
    tc::tmem_ld16(taddr + c, lead);
    tc::tmem_ld16(taddr + kBig + c, corr);
#pragma unroll
    for (int v = 0; v < 4; ++v)
      *reinterpret_cast<float4*>(&S[r][c + 4 * v]) =
          make_float4(__uint_as_float(lead[4 * v]) + __uint_as_float(corr[4 * v]),
                      __uint_as_float(lead[4 * v + 1]) + __uint_as_float(corr[4 * v + 1]),
                      __uint_as_float(lead[4 * v + 2]) + __uint_as_float(corr[4 * v + 2]),
                      __uint_as_float(lead[4 * v + 3]) + __uint_as_float(corr[4 * v + 3]));
  }
  tc::fence_before();
  __syncthreads();
  const int64_t q = q0 + 4 * lane;
#pragma unroll
  for (int j = 0; j < kRowsPerWarp; ++j) {
    const int rr = warp + (kThreads / 32) * j;
    const int64_t p = p0 + rr;
    if (p < m) {
      const float4 dd = *reinterpret_cast<const float4*>(&S[rr][4 * lane]);
      float* dst = M + p * ldm + q;
      if (q + 3 < m && (!DIAG || q + 3 <= p)) {
        *reinterpret_cast<float4*>(dst) = make_float4(x[j].x - dd.x, x[j].y - dd.y, x[j].z - dd.z, x[j].w - dd.w);
      } else {
        const float de[4] = {dd.x, dd.y, dd.z, dd.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (q + e < m && (!DIAG || q + e <= p)) dst[e] = __ldcg(dst + e) - de[e];
      }
    }
  }
  __syncthreads();  // the staging area holds the next task's operand planes
}

// FINAL epilogue: acc (tile layout) -= D, through the staging area.
__device__ __forceinline__ void tc_sub_acc(float (&acc)[8][8], uint32_t tmem, TileCholSmem<float>& sm) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, quarter = warp & 3, half = warp >> 2;
  const int tx = tid & 15, ty = tid >> 4;
  const int r = quarter * 32 + lane;
  const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
  for (int g = 0; g < 2; ++g) {
    const int c = half * 64 + g * 32;
    uint32_t dv[32];
    tc::tmem_ld32(taddr + c, dv);
#pragma unroll
    for (int j = 0; j < 32; ++j) sm.ls[r][c + j] = __uint_as_float(dv[j]);
    tc::tmem_ld32(taddr + kBig + c, dv);
#pragma unroll
    for (int j = 0; j < 32; ++j) sm.ls[r][c + j] += __uint_as_float(dv[j]);
  }
  tc::fence_before();
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] -= sm.ls[ty + 16 * i][tx + 16 * j];
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
    k_chol_tiles(int64_t m, int64_t ldm, T* M, T* dinv, T* Uinv, const int4* __restrict__ tasks, int ntasks, int nb,
                 int* state, unsigned* ticket, Scalars* sc, unsigned char* planes) {
  extern __shared__ __align__(16) unsigned char chol_tiles_smem[];
  TileCholSmem<T>& sm = *reinterpret_cast<TileCholSmem<T>*>(chol_tiles_smem);
  const int tid = threadIdx.x;
  constexpr bool kTc = sizeof(T) == 4;  // FP32 factor: products on the tensor cores
  uint32_t tmem = 0, mma_parity = 0;
  if constexpr (kTc) {
    if (tid == 0) {
      tc::mbar_init(tc::smem_u32(&sm.mma_bar), 1);
      tc::mbar_init(tc::smem_u32(&sm.full_bar[0]), 1);
      tc::mbar_init(tc::smem_u32(&sm.full_bar[1]), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((tid >> 5) == 0) tc::tmem_alloc(tc::smem_u32(&sm.tmem_slot), kTcCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    tmem = sm.tmem_slot;
  }
  int chain_step = 0;  // block 0: step 2 l is FINAL(l, l), step 2 l + 1 the solve of tile (l + 1, l)
  for (;;) {
    if (tid == 0) {  // take a task and wait for the tiles it starts from
      int go = 0;
      bool have = false;
      int4 d = make_int4(0, 0, 0, 0);
      if (blockIdx.x == 0) {  // the diagonal chain in order
        const int l = chain_step >> 1;
        if (chain_step & 1) {
          have = l + 1 < nb;
          d = make_int4(TK_CHAIN_SOLVE, l + 1, l, l);
        } else {
          have = l < nb;
          d = make_int4(TK_FINAL_DIAG, l, l, l - 1);
        }
        ++chain_step;
      } else {  // the other tasks in list order
        for (;;) {
          const unsigned t = atomicAdd(ticket, 1u);
          if (t >= (unsigned)ntasks) break;
          d = tasks[t];
          if (d.x != TK_FINAL_DIAG && d.x != TK_CHAIN_SOLVE) {
            have = true;
            break;
          }
        }
      }
      if (have && !dev_failed(sc)) {
        sm.task = d;
        const int64_t i = d.y, l = d.z, k = d.w;
        if (d.x == TK_UPDATE)
          go = wait_at_least(state + i * nb + k, (int)k + 1, sc) && wait_at_least(state + l * nb + k, (int)k + 1, sc) &&
               wait_at_least(state + i * nb + l, (int)k, sc);
        else if (d.x == TK_INV)
          go = wait_at_least(state + l * nb + l, (int)l + 1, sc);
        else if (d.x == TK_CHAIN_SOLVE)  // every update of the tile applied (L_ll is this block's own)
          go = wait_at_least(state + i * nb + l, (int)l, sc);
        else if (l == 0)
          go = 1;
        else
          go = wait_at_least(state + i * nb + l - 1, (int)l, sc) && wait_at_least(state + l * nb + l - 1, (int)l, sc) &&
               wait_at_least(state + i * nb + l, (int)l - 1, sc);
      }
      sm.go = go;
    }
    __syncthreads();
    if (!sm.go) break;
    const int4 d = sm.task;
    const int i = d.y, l = d.z;
    const int64_t p0 = (int64_t)i * kBig, q0 = (int64_t)l * kBig;
    T acc[8][8];
    int val;
    if (d.x == TK_INV) {  // (the double-float factor's solves substitute: no inverses)
      if constexpr (!std::is_same<T, dfloat>::value) tile_inverse<T>(acc, m, ldm, M, dinv, Uinv, l, sm);
      __syncthreads();  // (shared memory is reused by the next task; no counter to publish)
      continue;
    }
    if (d.x == TK_CHAIN_SOLVE) {  // block 0, right after FINAL(l, l): L_ll and 1 / L_cc are still in shared memory
      load_tile(acc, M, ldm, m, p0, q0, false);
      trsm_sweep<T>(acc, sm);
      store_tile(acc, M, ldm, m, p0, q0, false);
      if constexpr (kTc) tc_write_planes(acc, planes + plane_slot(i, l) * kTcTileBytes, sm);
      __threadfence();
      __syncthreads();
      if (tid == 0) st_release(state + (int64_t)i * nb + l, l + 1);
      continue;
    }
    if (d.x == TK_UPDATE) {
      if constexpr (kTc) {
        if (i == l) tc_product_begin<true>(planes, plane_slot(i, d.w), plane_slot(i, d.w), sm, tmem, mma_parity, sc);
        else tc_product_begin<false>(planes, plane_slot(i, d.w), plane_slot(l, d.w), sm, tmem, mma_parity, sc);
        float4 cx[kRowsPerWarp];
        tc_load_rows(cx, m, ldm, M, p0, q0);
        if (!tc_product_end(sm, mma_parity, sc)) break;
        if (i == l) tc_sub_global<true>(cx, m, ldm, M, p0, q0, tmem, sm);
        else tc_sub_global<false>(cx, m, ldm, M, p0, q0, tmem, sm);
      } else {
        load_tile(acc, M, ldm, m, p0, q0, i == l);
        if (i == l) rank_update<T, true>(acc, m, ldm, M, i, l, d.w, sm);
        else rank_update<T, false>(acc, m, ldm, M, i, l, d.w, sm);
        store_tile(acc, M, ldm, m, p0, q0, i == l);
      }
      val = d.w + 1;
    } else if (d.x == TK_FINAL_DIAG) {
      if constexpr (kTc) {
        if (l > 0) {
          tc_product_begin<true>(planes, plane_slot(l, l - 1), plane_slot(l, l - 1), sm, tmem, mma_parity, sc);
          load_tile(acc, M, ldm, m, p0, p0, true);
          if (!tc_product_end(sm, mma_parity, sc)) break;
          tc_sub_acc(acc, tmem, sm);
        } else {
          load_tile(acc, M, ldm, m, p0, p0, true);
        }
      } else {
        load_tile(acc, M, ldm, m, p0, p0, true);
        if (l > 0) rank_update<T, true>(acc, m, ldm, M, l, l, l - 1, sm);
      }
      if (!tile_potrf<T>(acc, m, ldm, M, dinv, l, sm, sc)) break;
      val = l + 1;
    } else {
      if constexpr (kTc) {
        if (l > 0) {
          tc_product_begin<false>(planes, plane_slot(i, l - 1), plane_slot(l, l - 1), sm, tmem, mma_parity, sc);
          load_tile(acc, M, ldm, m, p0, q0, false);
          if (!tc_product_end(sm, mma_parity, sc)) break;
          tc_sub_acc(acc, tmem, sm);
        } else {
          load_tile(acc, M, ldm, m, p0, q0, false);
        }
      } else {
        load_tile(acc, M, ldm, m, p0, q0, false);
        if (l > 0) rank_update<T, false>(acc, m, ldm, M, i, l, l - 1, sm);
      }
      if (tid == 0) sm.go = wait_at_least(state + (int64_t)l * nb + l, l + 1, sc);  // L_ll
      __syncthreads();
      if (!sm.go) break;
      load_diag_factor<T>(m, ldm, M, dinv, l, sm);
      trsm_sweep<T>(acc, sm);
      store_tile(acc, M, ldm, m, p0, q0, false);
      if constexpr (kTc) tc_write_planes(acc, planes + plane_slot(i, l) * kTcTileBytes, sm);
      val = l + 1;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release(state + (int64_t)i * nb + l, val);
  }
  if constexpr (kTc) {  // every exit: all MMAs have completed (or drained after a timeout)
    tc::fence_before();
    __syncthreads();
    if ((tid >> 5) == 0) {
      tc::fence_after();
      tc::tmem_dealloc(tmem, kTcCols);
    }
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
// on nproc identical workers.  Costs are per task kind, in microseconds as
// measured on GB300 for the FP32 factor (one CTA per SM): an update on the
// tensor cores, diagonal or not, 7; the diagonal task's product and
// factorisation 35; the off-diagonal solve with its load of L_ll and the
// write of its BF16 planes 22; the inverse 20.
void chol_tile_tasks(int64_t m, int nproc, std::vector<int4>* out) {
  const int nb = (int)chol_tile_count(m);
  out->clear();
  if (nb <= 0 || nb > kTileCholMaxTiles) return;
  if (nproc < 1) nproc = 1;
  constexpr double kUpd = 7.0, kUpdDiag = 7.0, kPotrf = 27.0, kTrsm = 22.0, kChain = 19.0, kInv = 20.0;
  struct Node {
    int4 d;
    double pre, post;  // cost before / after the mid-task wait (FINAL(i, l): for L_ll)
    int mid;           // FINAL(l, l) for FINAL(i, l), i > l + 1; else -1
    int npred;
  };
  std::vector<Node> nodes;
  std::vector<std::vector<int>> succ;
  // index maps: the task that finishes tile (i, l) -> fidx[i nb + l]; UPDATE(i, l, k) with
  // k <= l - 2 -> ubase[l nb + k] + i - l, and UPDATE(l + 1, l, l - 1) -> subupd[l]
  std::vector<int> fidx((size_t)nb * nb, -1), ubase((size_t)nb * nb, -1), subupd(nb, -1);
  auto add = [&](int4 d, double pre, double post) {
    nodes.push_back(Node{d, pre, post, -1, 0});
    return (int)nodes.size() - 1;
  };
  for (int l = 0; l < nb; ++l) {
    fidx[(size_t)l * nb + l] = add(make_int4(TK_FINAL_DIAG, l, l, l - 1), (l ? kUpdDiag : 0.0) + kPotrf, 0.0);
    add(make_int4(TK_INV, l, l, 0), kInv, 0.0);
    if (l + 1 < nb) fidx[(size_t)(l + 1) * nb + l] = add(make_int4(TK_CHAIN_SOLVE, l + 1, l, l), kChain, 0.0);
    for (int i = l + 2; i < nb; ++i) fidx[(size_t)i * nb + l] = add(make_int4(TK_FINAL_OFF, i, l, l - 1), l ? kUpd : 0.0, kTrsm);
    for (int k = 0; k + 2 <= l; ++k) {
      ubase[(size_t)l * nb + k] = (int)nodes.size();
      for (int i = l; i < nb; ++i) add(make_int4(TK_UPDATE, i, l, k), i == l ? kUpdDiag : kUpd, 0.0);
    }
    if (l >= 1 && l + 1 < nb) subupd[l] = add(make_int4(TK_UPDATE, l + 1, l, l - 1), kUpd, 0.0);
  }
  succ.resize(nodes.size());
  auto edge = [&](int a, int b) {
    succ[a].push_back(b);
    ++nodes[b].npred;
  };
  auto upd = [&](int i, int l, int k) { return k == l - 1 ? subupd[l] : ubase[(size_t)l * nb + k] + (i - l); };
  for (int v = 0; v < (int)nodes.size(); ++v) {
    const int4 d = nodes[v].d;
    const int i = d.y, l = d.z, k = d.w;
    if (d.x == TK_INV) {
      edge(fidx[(size_t)l * nb + l], v);
    } else if (d.x == TK_UPDATE) {
      edge(fidx[(size_t)i * nb + k], v);
      if (l != i) edge(fidx[(size_t)l * nb + k], v);
      if (k > 0) edge(upd(i, l, k - 1), v);
    } else if (d.x == TK_CHAIN_SOLVE) {  // every update of (l + 1, l) applied, L_ll final
      edge(fidx[(size_t)l * nb + l], v);
      if (l >= 1) edge(upd(i, l, l - 1), v);
    } else {
      if (l > 0) {
        edge(fidx[(size_t)i * nb + l - 1], v);
        if (i != l) edge(fidx[(size_t)l * nb + l - 1], v);
        if (l >= 2) edge(upd(i, l, l - 2), v);
      }
      if (d.x == TK_FINAL_OFF) nodes[v].mid = fidx[(size_t)l * nb + l];
    }
  }
  // bottom levels, over a topological order of the start and mid edges
  const int N = (int)nodes.size();
  std::vector<std::vector<int>> midsucc(N);
  for (int v = 0; v < N; ++v)
    if (nodes[v].mid >= 0) midsucc[nodes[v].mid].push_back(v);
  std::vector<int> indeg(N, 0), topo;
  topo.reserve(N);
  for (int v = 0; v < N; ++v) {
    for (int w : succ[v]) ++indeg[w];
    for (int w : midsucc[v]) ++indeg[w];
  }
  for (int v = 0; v < N; ++v)
    if (indeg[v] == 0) topo.push_back(v);
  for (size_t h = 0; h < topo.size(); ++h) {
    const int v = topo[h];
    for (int w : succ[v])
      if (--indeg[w] == 0) topo.push_back(w);
    for (int w : midsucc[v])
      if (--indeg[w] == 0) topo.push_back(w);
  }
  std::vector<double> bl(N, 0.0);
  for (int h = (int)topo.size() - 1; h >= 0; --h) {
    const int v = topo[h];
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
                           int ntasks, int* state, unsigned* ticket, Scalars* sc, unsigned char* planes) {
  if (sizeof(T) == 4 && !planes && chol_tile_count(m) > 1) return cudaErrorInvalidValue;
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
  int grid = sms * per_sm;  // (at least 2: block 0 runs only the diagonal tasks)
  if (grid > ntasks) grid = ntasks;
  if (grid < 2) return cudaErrorInvalidConfiguration;
  k_chol_tiles<T><<<grid, kThreads, chol_tiles_smem_bytes<T>(), st>>>(m, ldm, M, dinv, Uinv, tasks, ntasks, nb,
                                                                     state, ticket, sc, planes);
  return cudaGetLastError();
}

template cudaError_t cholesky_tiles<float>(cudaStream_t, int64_t, int64_t, float*, float*, float*, const int4*, int,
                                           int*, unsigned*, Scalars*, unsigned char*);
template cudaError_t cholesky_tiles<double>(cudaStream_t, int64_t, int64_t, double*, double*, double*, const int4*,
                                            int, int*, unsigned*, Scalars*, unsigned char*);

template cudaError_t cholesky_tiles<dfloat>(cudaStream_t, int64_t, int64_t, dfloat*, dfloat*, dfloat*, const int4*,
                                            int, int*, unsigned*, Scalars*, unsigned char*);

namespace {

// The lower triangle of the FP64 matrix M (leading dimension ldm) as
// double-float pairs in place (each 8-byte entry becomes hi, lo), or back.
__global__ void k_df_convert(int64_t m, int64_t ldm, double* M, int to_df) {
  const int64_t total = m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / m, q = e % m;
    if (q > p) continue;
    double* a = M + p * ldm + q;
    if (to_df) {
      const dfloat v = df_from_double(*a);
      *reinterpret_cast<float2*>(a) = make_float2(v.hi, v.lo);
    } else {
      const float2 v = *reinterpret_cast<const float2*>(a);
      *a = df_to_double(dfloat(v.x, v.y));
    }
  }
}
__global__ void k_df_to_double(int64_t n, double* v) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const float2 w = *reinterpret_cast<const float2*>(v + j);
    v[j] = df_to_double(dfloat(w.x, w.y));
  }
}

}  // namespace

cudaError_t cholesky_tiles_df(cudaStream_t st, int64_t m, int64_t ldm, double* M, double* dinv, const int4* tasks,
                              int ntasks, int* state, unsigned* ticket, Scalars* sc) {
  const unsigned g = (unsigned)std::min<int64_t>((m * m + 255) / 256, 4736);
  k_df_convert<<<g, 256, 0, st>>>(m, ldm, M, 1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cholesky_tiles<dfloat>(st, m, ldm, reinterpret_cast<dfloat*>(M), reinterpret_cast<dfloat*>(dinv), nullptr,
                               tasks, ntasks, state, ticket, sc, nullptr);
  if (e != cudaSuccess) return e;
  k_df_convert<<<g, 256, 0, st>>>(m, ldm, M, 0);
  k_df_to_double<<<(unsigned)std::min<int64_t>((m + 255) / 256, 1184), 256, 0, st>>>(m, dinv);
  return cudaGetLastError();
}

int64_t chol_plane_bytes(int64_t m) {
  const int64_t nb = chol_tile_count(m);
  return nb * (nb - 1) / 2 * kTcTileBytes;
}

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
