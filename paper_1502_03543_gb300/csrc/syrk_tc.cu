// syrk_tc.cu -- the normal matrix M = A D A' (Section V) on the tcgen05
// tensor cores, for the BF16 and TF32 mixed-precision forms.
//
// TF32 form (A stored in FP64 or FP32): A and B = D.*A are rounded once per
// call to TF32 (FP32 containers, 10 stored mantissa bits, round to nearest
// even) and M = A_tf32 B_tf32' takes one tcgen05.mma.kind::tf32 term; each
// operand carries 2^-11 relative error, which the FP64 refinement removes
// from the direction.  With three terms (TF32 x 3) both operands are split,
// A = A_0 + A_1 and B = B_0 + B_1 (hi and lo TF32 parts, ~2^-22 relative
// left over), and M ~= A_0 B_0' + A_0 B_1' + A_1 B_0': every product is exact
// in FP32, so M is FP32-grade.  The rest of this header describes the BF16
// form; the TF32 kernel is the same pipeline with 32 FP32 elements per
// 128-byte row.
//
// D is folded into one operand: B = D.*A (row q: B_qj = A_qj D_j) is split
// into `splits` BF16 terms B = B_0 + B_1 (+ B_2), each carrying the next 8
// bits of the FP32 product, so every product A_pj B_t,qj is exact and
//     M ~= sum_t A B_t'.
// A (BF16, exact) is read in place by TMA when its rows are 16-byte aligned.
//
// Accumulation.  The tensor core's FP32 accumulator rounds toward zero, so
// its error grows with the number of accumulation steps in one direction
// (measured on GB300: 1.5e-4 relative at K = 32768 against 1e-6 for an IEEE
// FP32 dot product).  The K loop is therefore cut into chunks of KC = 128
// elements (64 for TF32): each chunk is summed on the tensor core into a
// fresh TMEM buffer (two buffers alternate), and the epilogue warps add the
// chunk sums, with round-to-nearest FP32, into a master accumulator held in
// registers.
//
// Kernel k_syrk_tc<S, TF32, ALO>: one CTA per 128 x 128 lower-triangle tile,
// 6 warps:
//   warp 0      TMA producer: per K step of one 128-byte swizzle row (64 BF16
//               or 32 TF32 elements) the A tile (and A_1 for TF32 x 3) and
//               the S tiles of B_t, 16 KB each, into a ring of
//               STAGES (= 192 KB / (16 KB x tiles per stage)) stages;
//   warp 1      allocates 256 TMEM columns; one lane issues
//               tcgen05.mma.cta_group::1.kind::f16 (M=128, N=128, K=16) or
//               .kind::tf32 (K=8), four per product and K step, into the
//               current chunk buffer and commits chunk and stage;
//   warps 2..5  warp w owns TMEM lanes 32*(w%4)..: drains each chunk
//               (tcgen05.ld) into its 128-float master row, frees the
//               buffer, and finally writes the rows p >= q of M.
// Every mbarrier wait is bounded (2 s); on a timeout the CTA sets
// PDAS_ERR_TIMEOUT, drains its in-flight copies and MMAs, frees TMEM, exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <new>
#include <vector>

#include "syrk_tc.cuh"
#include "tc_util.cuh"

namespace pdas {

namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 64;        // K elements of one 128-byte operand row (BF16)
constexpr int BK_TF32 = 32;   // the same for TF32 (4-byte containers)
constexpr int KC_BLOCKS = 2;  // K steps of BK per accumulation chunk (KC = 128)
constexpr uint32_t TILE_BYTES = BM * 128;     // one 128-row x 128-byte tile (A and each B_t)
constexpr uint32_t RING_BYTES = 192 * 1024;
constexpr uint32_t TMEM_COLS = 256;           // two chunk buffers of BN columns
constexpr int NUM_THREADS = 192;
constexpr size_t SMEM_BYTES = 1024 + (size_t)RING_BYTES + 512;

template <int TILES>  // operand tiles per stage
struct Ring {
  static constexpr uint32_t STAGE_BYTES = TILE_BYTES * TILES;
  static constexpr int STAGES = (int)(RING_BYTES / STAGE_BYTES);
};

using namespace tc;
constexpr uint32_t kIdescBf16 = idesc_bf16(BM, BN);
constexpr uint32_t kIdescTf32 = idesc_tf32(BM, BN);

// S terms B_t of D.*A.  ALO (TF32 x 3): A = A_0 + A_1 in two planes as well,
// S = 2, the stage holds A_0 | B_0 | B_1 | A_1 (A_1 through the tmB2 map) and
// the products are A_0 B_0' + A_0 B_1' + A_1 B_0' (A_1 B_1' is below the
// rounding of the rest).
template <int S, bool TF32 = false, bool ALO = false>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_syrk_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB0,
              const __grid_constant__ CUtensorMap tmB1, const __grid_constant__ CUtensorMap tmB2,
              const int2* __restrict__ tiles, int nk, int64_t m, int64_t ldm, float* __restrict__ M, Scalars* sc) {
  static_assert(!ALO || S == 2, "the split-A form pairs two planes of A with two of D.*A");
  constexpr uint32_t STAGE_BYTES = Ring<1 + S + (ALO ? 1 : 0)>::STAGE_BYTES;
  constexpr int STAGES = Ring<1 + S + (ALO ? 1 : 0)>::STAGES;
  constexpr int NP = ALO ? 3 : S;  // MMA products per K step
  constexpr int EK = TF32 ? BK_TF32 : BK;  // K elements per stage
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RING_BYTES);
  // bars: full[STAGES] | empty[STAGES] | chunk_full[2] | chunk_free[2] | done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + STAGES + s); };
  auto chunk_full = [&](int b) { return smem_u32(bars + 2 * STAGES + b); };
  auto chunk_free = [&](int b) { return smem_u32(bars + 2 * STAGES + 2 + b); };
  const uint32_t done_bar = smem_u32(bars + 2 * STAGES + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int2 tile = tiles[blockIdx.x];
  const int p0 = tile.x * BM, q0 = tile.y * BN;
  const int nchunks = (nk + KC_BLOCKS - 1) / KC_BLOCKS;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(chunk_full(b), 1);
      mbar_init(chunk_free(b), 4);  // one arrival per epilogue warp
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
        if (!mbar_wait(empty(s), ph ^ 1u, abort_flag)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t dst = sbase + s * STAGE_BYTES;
        mbar_expect_tx(full(s), STAGE_BYTES);
        tma_load_2d(dst, &tmA, kb * EK, p0, full(s));
        tma_load_2d(dst + TILE_BYTES, &tmB0, kb * EK, q0, full(s));
        if (S > 1) tma_load_2d(dst + 2 * TILE_BYTES, &tmB1, kb * EK, q0, full(s));
        if (S > 2) tma_load_2d(dst + 3 * TILE_BYTES, &tmB2, kb * EK, q0, full(s));
        if (ALO) tma_load_2d(dst + (1 + S) * TILE_BYTES, &tmB2, kb * EK, p0, full(s));  // A_1
        issued = kb + 1;
      }
      if (*abort_flag) {  // let every issued copy land before the CTA can exit
        for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
          mbar_wait(full(kb % STAGES), (uint32_t)(kb / STAGES) & 1u, nullptr);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      for (int kb = 0; kb < nk && !*abort_flag; ++kb) {
        const int c = kb / KC_BLOCKS, buf = c & 1;
        const bool chunk_start = (kb % KC_BLOCKS) == 0;
        if (chunk_start && c >= 2 &&
            !mbar_wait(chunk_free(buf), (uint32_t)((c >> 1) - 1) & 1u, abort_flag)) {
          *abort_flag = 1;
          break;
        }
        const int s = kb % STAGES;
        if (!mbar_wait(full(s), (uint32_t)(kb / STAGES) & 1u, abort_flag)) {
          *abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * BN);
#pragma unroll
        for (int t = 0; t < NP; ++t) {
          const int ia = (ALO && t == 2) ? 1 + S : 0;      // tile of A_0 or A_1
          const int ib = 1 + ((ALO && t == 2) ? 0 : t);   // tile of B_t
          const uint64_t ad = sdesc_sw128(sbase + s * STAGE_BYTES + ia * TILE_BYTES);
          const uint64_t bd = sdesc_sw128(sbase + s * STAGE_BYTES + ib * TILE_BYTES);
#pragma unroll
          for (int k = 0; k < 4; ++k) {  // advance 32 bytes (16 BF16 or 8 TF32) along K per MMA
            const uint32_t accum = (chunk_start && t == 0 && k == 0) ? 0u : 1u;
            if constexpr (TF32) umma_tf32(d, ad + 2 * k, bd + 2 * k, kIdescTf32, accum);
            else umma_f16(d, ad + 2 * k, bd + 2 * k, kIdescBf16, accum);
          }
        }
        umma_commit(empty(s));
        if ((kb % KC_BLOCKS) == KC_BLOCKS - 1 || kb == nk - 1) umma_commit(chunk_full(buf));
      }
      umma_commit(done_bar);  // fires once every MMA issued above has completed
      mbar_wait(done_bar, 0, nullptr);
    }
    __syncwarp();
  } else {
    const int quarter = warp & 3;  // TMEM lanes this warp may read
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    float acc[BN];
#pragma unroll
    for (int j = 0; j < BN; ++j) acc[j] = 0.f;
    int ok = 1;
    for (int c = 0; c < nchunks; ++c) {
      const int buf = c & 1;
      if (lane == 0) ok = mbar_wait(chunk_full(buf), (uint32_t)(c >> 1) & 1u, abort_flag) && !*abort_flag;
      ok = __shfl_sync(0xffffffffu, ok, 0);  // warp-uniform for tcgen05.ld
      if (!ok) break;
      fence_after();
#pragma unroll
      for (int g = 0; g < BN / 32; ++g) {
        uint32_t r[32];
        tmem_ld32(lane_addr + (uint32_t)(buf * BN + g * 32), r);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[g * 32 + j] += __uint_as_float(r[j]);  // round to nearest
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(chunk_free(buf));
    }
    if (ok) {
      const int64_t p = p0 + quarter * 32 + lane;
      if (p < m) {
        float* dst = M + p * ldm;
#pragma unroll
        for (int j = 0; j < BN; ++j) {
          const int64_t q = (int64_t)q0 + j;
          if (q <= p) dst[q] = acc[j];
        }
      }
    } else if (lane == 0) {
      *abort_flag = 1;
    }
  }
  if (threadIdx.x == 0 && *abort_flag) atomicCAS(&sc->status, 0, (int)PDAS_ERR_TIMEOUT);
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// D32 = (float) D.
__global__ void k_d32(int64_t n, const double* __restrict__ D, float* __restrict__ D32) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    D32[j] = (float)D[j];
}

// Split B = D.*A into BF16 terms: v = A_pj * D_j in FP32; B_0 = bf16(v),
// B_1 = bf16(v - B_0), B_2 = bf16(v - B_0 - B_1) (each difference exact in
// FP32).  opb holds `splits` planes of m rows x kpad; opa, if given, receives
// a copy of A with row stride kpad (rows of A not 16-byte aligned).
__global__ void k_fold_split(int64_t m, int64_t n, int64_t kpad, const __nv_bfloat16* __restrict__ A,
                             const float* __restrict__ D32, int splits, __nv_bfloat16* __restrict__ opb,
                             __nv_bfloat16* __restrict__ opa, int vec) {
  const int64_t plane = m * kpad;
  if (vec) {
    const int64_t groups_per_row = n / 8;
    const int64_t total = m * groups_per_row;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
      const int64_t p = g / groups_per_row, j = (g % groups_per_row) * 8;
      const uint4 raw = __ldg(reinterpret_cast<const uint4*>(A + p * n + j));
      const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
      const float4 d0 = __ldg(reinterpret_cast<const float4*>(D32 + j));
      const float4 d1 = __ldg(reinterpret_cast<const float4*>(D32 + j + 4));
      const float dd[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
      uint32_t out[3][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float v[2] = {__uint_as_float(w[i] << 16) * dd[2 * i], __uint_as_float(w[i] & 0xffff0000u) * dd[2 * i + 1]};
        uint16_t h[3][2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          float rest = v[e];
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            const __nv_bfloat16 b = __float2bfloat16_rn(rest);
            h[t][e] = __bfloat16_as_ushort(b);
            rest = rest - __bfloat162float(b);
          }
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) out[t][i] = (uint32_t)h[t][0] | ((uint32_t)h[t][1] << 16);
      }
      for (int t = 0; t < splits; ++t)
        *reinterpret_cast<uint4*>(opb + t * plane + p * kpad + j) = make_uint4(out[t][0], out[t][1], out[t][2],
                                                                               out[t][3]);
      if (opa) *reinterpret_cast<uint4*>(opa + p * kpad + j) = raw;
    }
  } else {
    const int64_t total = m * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t p = e / n, j = e % n;
      const __nv_bfloat16 a = A[e];
      float rest = __bfloat162float(a) * D32[j];
      for (int t = 0; t < splits; ++t) {
        const __nv_bfloat16 b = __float2bfloat16_rn(rest);
        opb[t * plane + p * kpad + j] = b;
        rest = rest - __bfloat162float(b);
      }
      if (opa) opa[p * kpad + j] = a;
    }
  }
}

// Round an FP32 value to TF32 (10 stored mantissa bits), to nearest with ties
// to even: add one less than half the spacing of the TF32 grid, plus the
// lowest kept bit, then clear the 13 dropped bits.  Inf stays inf, a finite
// value above the largest TF32 number rounds to inf.
__device__ __forceinline__ float round_tf32(float f) {
  uint32_t u = __float_as_uint(f);
  u += 0xfffu + ((u >> 13) & 1u);
  return __uint_as_float(u & 0xffffe000u);
}

// TF32 operands: opa = tf32(A), opb = tf32(fl32(A_pj D_j)) with the product in
// FP64 (exact for FP32 A), both with row stride kpad.  split: a second plane
// of each (at plane stride m kpad) takes the rest, tf32(fl32(v) - tf32(fl32(v)))
// (the difference is exact in FP32).
template <typename T>
__global__ void k_fold_tf32(int64_t m, int64_t n, int64_t kpad, const T* __restrict__ A,
                            const double* __restrict__ D, float* __restrict__ opa, float* __restrict__ opb,
                            int split) {
  const int64_t total = m * n, plane = m * kpad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / n, j = e - p * n, o = p * kpad + j;
    const double a = (double)A[e];
    const float a32 = (float)a, b32 = (float)(a * D[j]);
    const float a0 = round_tf32(a32), b0 = round_tf32(b32);
    opa[o] = a0;
    opb[o] = b0;
    if (split) {
      opa[plane + o] = round_tf32(a32 - a0);
      opb[plane + o] = round_tf32(b32 - b0);
    }
  }
}

// ---- host side ---------------------------------------------------------------
struct TcHost {
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  CUtensorMap mapB[3];
  CUtensorMap mapA_copy;
  int2* tiles = nullptr;
  int ntiles = 0;
  float* D32 = nullptr;
  bool smem_attr_set = false;
};

cudaError_t get_encoder(PFN_cuTensorMapEncodeTiled_v12000* out) {
  static std::mutex mu;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  *out = fn;
  return cudaSuccess;
}

// 2D BF16 (or, with tf32, FP32) tensor map: dims {n (K, innermost), m}, row
// stride in elements, box {one 128-byte row, box_rows}, 128-byte swizzle,
// zero fill out of bounds.
cudaError_t encode_bf16(TcHost* hs, CUtensorMap* map, const void* base, int64_t m, int64_t n, int64_t row_stride,
                        int box_rows, bool tf32 = false) {
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
  cuuint64_t strides[1] = {(cuuint64_t)(row_stride * (tf32 ? 4 : 2))};
  cuuint32_t box[2] = {(cuuint32_t)(tf32 ? BK_TF32 : BK), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = hs->encode(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                          const_cast<void*>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t tc_workspace_create(TcWorkspace* w, int form, int a_dtype, int splits, int64_t m, int64_t n) {
  const bool tf32 = form == PDAS_TF32_IR;
  if (tf32 ? (a_dtype != PDAS_A_F64 && a_dtype != PDAS_A_F32) || splits == 2 || splits > 3
           : (form != PDAS_BF16_IR || a_dtype != PDAS_A_BF16))
    return cudaErrorNotSupported;
  if (m > ((int64_t)1 << 30) / BM || n > ((int64_t)1 << 31) - BK) return cudaErrorNotSupported;
  w->form = form;
  w->a_dtype = a_dtype;
  w->splits = tf32 ? (splits == 1 ? 1 : 3) : splits > 0 ? splits : 3;
  w->m = m;
  w->n = n;
  w->kpad = (n + BK - 1) / BK * BK;
  w->mpad = (m + BN - 1) / BN * BN;
  TcHost* hs = new (std::nothrow) TcHost();
  if (!hs) return cudaErrorMemoryAllocation;
  w->host = hs;
  cudaError_t e = get_encoder(&hs->encode);
  if (e != cudaSuccess) return e;
  const size_t esz = tf32 ? sizeof(float) : sizeof(__nv_bfloat16);
  // planes: BF16, splits terms of D.*A (and a padded copy of A if its rows are
  // not 16-byte aligned); TF32, one plane of each operand, or two (TF32 x 3)
  const int bplanes = tf32 ? (w->splits == 3 ? 2 : 1) : w->splits;
  const int aplanes = tf32 ? bplanes : 1;
  e = cudaMalloc(&w->opb, esz * (size_t)bplanes * m * w->kpad);
  if (e == cudaSuccess && (tf32 || n % 8 != 0)) e = cudaMalloc(&w->opa, esz * (size_t)aplanes * m * w->kpad);
  if (e == cudaSuccess) e = cudaMalloc(&hs->D32, sizeof(float) * (size_t)((n + 7) / 8 * 8));
  // Lower-triangle tile list ((I, J) with some row p >= some column q),
  // ordered by G x G super-tiles with G ~ sqrt(#SMs): the CTAs resident at
  // one time then cover about G row blocks of A and G row blocks of the
  // split planes, whose K panels they stream at roughly the same pace, so L2
  // serves most operand reads (in plain row order a wave spans a few rows of
  // tiles but up to all tile columns, and the split planes were re-read from
  // DRAM about a dozen times per launch).  Super-tiles go in row-major lower
  // order, so consecutive ones share their row blocks of A.
  std::vector<int2> tl;
  const int64_t nI = (m + BM - 1) / BM, nJ = (m + BN - 1) / BN;
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t G = 1;
  while ((G + 1) * (G + 1) <= (int64_t)sms) ++G;
  for (int64_t PI = 0; PI < nI; PI += G)
    for (int64_t PJ = 0; PJ <= PI; PJ += G)
      for (int64_t I = PI; I < nI && I < PI + G; ++I)
        for (int64_t J = PJ; J < nJ && J < PJ + G && J * BN <= I * BM + BM - 1; ++J)
          tl.push_back(make_int2((int)I, (int)J));
  hs->ntiles = (int)tl.size();
  if (e == cudaSuccess) e = cudaMalloc(&hs->tiles, sizeof(int2) * tl.size());
  if (e == cudaSuccess) e = cudaMemcpy(hs->tiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice);
  for (int t = 0; e == cudaSuccess && t < 3; ++t) {
    const int tt = t < bplanes ? t : 0;  // unused maps alias term 0
    if (tf32 && bplanes == 2 && t == 2)  // TF32 x 3: the third map carries A_1
      e = encode_bf16(hs, &hs->mapB[t], (const uint8_t*)w->opa + esz * m * w->kpad, m, n, w->kpad, BM, tf32);
    else
      e = encode_bf16(hs, &hs->mapB[t], (const uint8_t*)w->opb + esz * tt * m * w->kpad, m, n, w->kpad, BN, tf32);
  }
  if (e == cudaSuccess && w->opa) e = encode_bf16(hs, &hs->mapA_copy, w->opa, m, n, w->kpad, BM, tf32);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_syrk_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_syrk_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_syrk_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_syrk_tc<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_syrk_tc<2, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
  return e;
}

void tc_workspace_destroy(TcWorkspace* w) {
  if (w->opa) cudaFree(w->opa);
  if (w->opb) cudaFree(w->opb);
  TcHost* hs = static_cast<TcHost*>(w->host);
  if (hs) {
    if (hs->tiles) cudaFree(hs->tiles);
    if (hs->D32) cudaFree(hs->D32);
    delete hs;
  }
  *w = TcWorkspace{};
}

cudaError_t tc_prepare(cudaStream_t st, TcWorkspace* w, const void* A, const double* D, int* launches) {
  *launches = 0;
  if (reinterpret_cast<uintptr_t>(A) % 16 != 0) return cudaErrorInvalidValue;
  TcHost* hs = static_cast<TcHost*>(w->host);
  const int64_t m = w->m, n = w->n;
  if (w->form == PDAS_TF32_IR) {
    const int64_t work = m * n;
    const unsigned grid = (unsigned)((work + 255) / 256 < 4736 ? (work + 255) / 256 : 4736);
    const int split = w->splits == 3 ? 1 : 0;
    if (w->a_dtype == PDAS_A_F64)
      k_fold_tf32<double><<<grid, 256, 0, st>>>(m, n, w->kpad, static_cast<const double*>(A), D,
                                                static_cast<float*>(w->opa), static_cast<float*>(w->opb), split);
    else
      k_fold_tf32<float><<<grid, 256, 0, st>>>(m, n, w->kpad, static_cast<const float*>(A), D,
                                               static_cast<float*>(w->opa), static_cast<float*>(w->opb), split);
    *launches = 1;
    return cudaGetLastError();
  }
  const bool direct = (n % 8 == 0);
  k_d32<<<(unsigned)((n + 255) / 256 < 1184 ? (n + 255) / 256 : 1184), 256, 0, st>>>(n, D, hs->D32);
  const int64_t work = direct ? m * (n / 8) : m * n;
  unsigned grid = (unsigned)((work + 255) / 256 < 4736 ? (work + 255) / 256 : 4736);
  if (grid < 1) grid = 1;
  k_fold_split<<<grid, 256, 0, st>>>(m, n, w->kpad, static_cast<const __nv_bfloat16*>(A), hs->D32, w->splits,
                                     static_cast<__nv_bfloat16*>(w->opb),
                                     direct ? nullptr : static_cast<__nv_bfloat16*>(w->opa), direct ? 1 : 0);
  *launches = 2;
  return cudaGetLastError();
}

cudaError_t tc_syrk(cudaStream_t st, TcWorkspace* w, const void* A, float* M32, int64_t ldm, const Scalars* sc,
                    int* launches) {
  *launches = 0;
  TcHost* hs = static_cast<TcHost*>(w->host);
  const int64_t m = w->m, n = w->n;
  Scalars* scw = const_cast<Scalars*>(sc);
  const dim3 grid((unsigned)hs->ntiles);
  if (w->form == PDAS_TF32_IR) {
    const int nk = (int)((n + BK_TF32 - 1) / BK_TF32);
    if (w->splits == 3)
      k_syrk_tc<2, true, true><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(hs->mapA_copy, hs->mapB[0], hs->mapB[1],
                                                                      hs->mapB[2], hs->tiles, nk, m, ldm, M32, scw);
    else
      k_syrk_tc<1, true><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(hs->mapA_copy, hs->mapB[0], hs->mapB[1],
                                                                hs->mapB[2], hs->tiles, nk, m, ldm, M32, scw);
    *launches = 1;
    return cudaGetLastError();
  }
  CUtensorMap mapA;
  if (n % 8 == 0) {
    cudaError_t e = encode_bf16(hs, &mapA, A, m, n, n, BM);
    if (e != cudaSuccess) return e;
  } else {
    mapA = hs->mapA_copy;
  }
  const int nk = (int)((n + BK - 1) / BK);
  if (w->splits == 1)
    k_syrk_tc<1><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(mapA, hs->mapB[0], hs->mapB[1], hs->mapB[2], hs->tiles, nk,
                                                        m, ldm, M32, scw);
  else if (w->splits == 2)
    k_syrk_tc<2><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(mapA, hs->mapB[0], hs->mapB[1], hs->mapB[2], hs->tiles, nk,
                                                        m, ldm, M32, scw);
  else
    k_syrk_tc<3><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(mapA, hs->mapB[0], hs->mapB[1], hs->mapB[2], hs->tiles, nk,
                                                        m, ldm, M32, scw);
  *launches = 1;
  return cudaGetLastError();
}

}  // namespace pdas
