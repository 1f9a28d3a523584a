// syrk_dig.cu -- the FP64 tier's normal matrix M = A D A' (Section V) on the
// tcgen05 tensor cores, for A stored in BF16, to FP64-grade accuracy.
//
// Why: once the FP32 factor of a mixed form breaks down (cond(A D A') beyond
// FP32), the solve needs an FP64-grade M of the kept columns every
// iteration.  On GB300 FP64 runs at 1/64 of the FP32 rate and the FP32-pipe
// double-float SYRK does ~10 operations per term; both are far below what
// the BF16 tensor cores give.  Here the products are made exact and the
// accumulation exact, so the tensor cores' FP32 accumulator loses nothing.
//
// Fixed-point digits.  Row p of A (kept columns j < k) is scaled by 2^-ea_p,
// ea_p the exponent of max_j |A_pj|, so a'_pj = A_pj 2^-ea_p lies in (-1, 1);
// row q of B = D.*A (B_qj = D_j A_qj, the exact integer product of the two
// significands) by 2^-eb_q.  Each is written in balanced base-256 digits:
//     a' = sum_{s<5} d_s 2^(-7-8s),    b' = sum_{t<8} g_t 2^(-7-8t),
// every digit an integer in [-128, 128] (exact in BF16).  Five digits hold a
// BF16 entry exactly down to 2^-32 of its row's largest; eight hold B to
// 2^-63.  Then
//     M_pq = 2^(ea_p + eb_q - 14) sum_w 2^(-8w) I_w,
//     I_w  = sum_j sum_{s+t=w} d_s,pj g_t,qj          (integers),
// for the 30 digit pairs with s + t <= 7 (the pairs dropped contribute at
// most 2^-62 of 2^(ea_p + eb_q) per column).  Every product d g has
// magnitude <= 2^14; a weight collects at most 5 pairs, so over a chunk of
// 192 columns |I_w| <= 5 * 192 * 2^14 < 2^24: the FP32 accumulator holds
// the chunk sum exactly, whatever its rounding.  The epilogue converts each
// chunk's weight sums to integers and adds them, weighted by powers of 2^8,
// exactly into int64 sums: hi (weights 0-3) and lo (weights 4-7).  At the
// end hi + 2^-32 lo is formed in FP64 and scaled by a power of two: the one
// rounding of an entry besides the digits' own truncation.
//
// The tensor cores read both operands of every MMA from shared memory, and
// that operand traffic bounded the kernel (the tc pipe, not the math, was
// 89 % busy at N = 32).  The tiles are therefore 128 rows p x 64 rows q, and
// the product runs in two passes so that one pass's weights fit tensor
// memory twice (2 chunk buffers x 4 weights x 64 columns = 512 columns) and
// its int64 sums fit the epilogue's registers: pass 0 forms the 10 pairs of
// weights 0-3 and leaves hi in M (int64 bits), pass 1 the 20 pairs of
// weights 4-7, reads hi back and writes M_pq.
//
// Kernel k_syrk_dig<pass>: one CTA per 128 x 64 lower-triangle tile, 10 warps:
//   warp 0      TMA producer: per stage of 32 columns one 3-D copy of the A
//               digit planes the pass needs (128 rows) and one of its B
//               planes (64 rows), 64-byte swizzle, 48 KB or 72 KB, into a
//               ring of 3 stages;
//   warp 1      allocates 512 TMEM columns; one lane issues
//               tcgen05.mma.cta_group::1.kind::f16 (M = 128, K = 16), 2 per
//               A digit per stage: the pairs (s, t) of A digit s in the pass
//               have consecutive t, so one MMA with N = 64 x (pairs) reads
//               the A plane once for all of them and writes the
//               accumulators of weights s + t, which lie one after another
//               in the current chunk buffer (4 or 5 MMAs per K step instead
//               of 10 or 20);
//   warps 2..9  warp w reads TMEM lanes 32 (w % 4).. and columns
//               32 ((w - 2) / 4).. of every weight: per chunk 4 x 32 values,
//               converted and added into int64 sums; then the buffer is
//               handed back.
// Every mbarrier wait is bounded (2 s); on a timeout the CTA sets
// PDAS_ERR_TIMEOUT, drains its in-flight copies and MMAs, frees TMEM, exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <mutex>
#include <vector>

#include "syrk_dig.cuh"
#include "tc_util.cuh"

namespace pdas {

namespace {

using namespace tc;

// 3-D tiled copy (coordinates innermost first) into shared memory; the box
// lands as dim2 x dim1 x dim0 contiguous, completing its bytes on bar.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* map, int c0, int c1, int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

constexpr int DBM = 128;                               // rows p of a tile (A digits)
constexpr int DBN = 64;                                // rows q of a tile (B digits)
constexpr int DBK = 64;                                // column granule of the planes (kfill, kstride)
constexpr int DSK = 32;                                // columns per stage (one 64-byte row)
constexpr int SA = 5, SB = 8, WMAX = 7;                // digits of A and B, largest pair weight kept
constexpr int NWP = 4;                                 // weights per pass: 0-3, then 4-7
constexpr int CHUNK_STAGES = 6;                        // 192 columns per exact chunk
constexpr uint32_t A_PLANE = DBM * DSK * 2;            // 8 KB: 128 rows of one digit, one stage
constexpr uint32_t B_PLANE = DBN * DSK * 2;            // 4 KB
constexpr uint32_t BUF_COLS = NWP * DBN;               // 256 TMEM columns per chunk buffer
constexpr uint32_t TMEM_COLS = 2 * BUF_COLS;           // 512
constexpr int NUM_THREADS = 320;

// The digit pairs (s, t) of a pass: weights W0 .. W0 + 3, s < SA, t < SB.
// Pass 0 (weights 0-3) has 10 pairs and reads A digits 0-3 and B digits 0-3;
// pass 1 (weights 4-7) has 20 pairs and reads all 13 planes.  A weight
// collects at most 5 pairs, so over a chunk of 192 columns
// |I_w| <= 5 * 192 * 2^14 < 2^24: exact in the FP32 accumulator.
template <int PASS>
struct DigPass {
  static constexpr int W0 = PASS * NWP;
  static constexpr int NA = PASS == 0 ? 4 : SA;  // A planes loaded
  static constexpr int NB = PASS == 0 ? 4 : SB;  // B planes loaded
  static constexpr uint32_t STAGE_BYTES = NA * A_PLANE + NB * B_PLANE;  // 48 KB or 72 KB
  // copies in flight: pass 0 has half the pairs per copied K step, so it
  // keeps one more stage in flight (4 x 48 KB; pass 1 3 x 72 KB)
  static constexpr int STAGES = PASS == 0 ? 4 : 3;
  static constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + 256;
  __host__ __device__ static constexpr bool kept(int s, int t) { return s + t >= W0 && s + t < W0 + NWP && s < NA && t < NB; }
  // the B digits t paired with A digit s in this pass: first_t(s) .. last_t(s)
  __host__ __device__ static constexpr int first_t(int s) { return W0 - s > 0 ? W0 - s : 0; }
  __host__ __device__ static constexpr int last_t(int s) { return W0 + NWP - 1 - s < NB - 1 ? W0 + NWP - 1 - s : NB - 1; }
};
// first_t .. last_t is exactly the pairs kept, at most 4 of them (N <= 256),
// and A digit 0 meets every weight of the pass
template <int PASS>
constexpr bool pass_groups_ok() {
  using P = DigPass<PASS>;
  if (P::first_t(0) != P::W0 || P::last_t(0) != P::W0 + NWP - 1) return false;
  for (int s = 0; s < P::NA; ++s) {
    if (P::last_t(s) - P::first_t(s) + 1 > 4) return false;
    for (int t = 0; t < P::NB; ++t)
      if (P::kept(s, t) != (t >= P::first_t(s) && t <= P::last_t(s))) return false;
  }
  return true;
}
static_assert(pass_groups_ok<0>() && pass_groups_ok<1>(), "one MMA per A digit covers the pass's pairs");
static_assert(5 * DSK * CHUNK_STAGES * 16384 < (1 << 24), "exact chunk");
static_assert(DigPass<0>::W0 + 2 * NWP - 1 == WMAX, "the two passes cover the weights 0..WMAX");
static_assert(DigPass<0>::SMEM_BYTES <= 232448 && DigPass<1>::SMEM_BYTES <= 232448, "shared memory of one CTA");

// Shared-memory matrix descriptor: K-major operand, rows of 64 bytes (32 BF16)
// with the 64-byte swizzle; 8-row groups 512 bytes apart (version 1 at bit
// 46, layout type 4 = 64-byte swizzle at bits 61-63).  Advancing the start
// address by 32 bytes moves one MMA step (16 BF16) along K.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address, 16-byte units
  d |= (uint64_t)1 << 16;                             // leading byte offset (unused when swizzled)
  d |= (uint64_t)(512 >> 4) << 32;                    // stride byte offset: one 8-row group
  d |= (uint64_t)1 << 46;                             // descriptor version
  d |= (uint64_t)4 << 61;                             // 64-byte swizzle
  return d;
}

// One pass of the digit product over the lower-triangle tiles (128 rows p x
// 64 rows q): pass 0 leaves hi = sum_{w<4} I_w 2^(8(3-w)) of every entry in
// M (its int64 bits), pass 1 forms lo = sum_{w>=4} I_w 2^(8(7-w)), reads hi
// back and writes M_pq = 2^(ea_p + eb_q - 38) (hi + 2^-32 lo) in FP64.
template <int PASS>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_syrk_dig(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const int2* __restrict__ tiles, int nk, int64_t m, const int* __restrict__ ea,
               const int* __restrict__ eb, int64_t ldm, double* __restrict__ M, Scalars* sc) {
  using P = DigPass<PASS>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + P::STAGES * P::STAGE_BYTES);
  // bars: full[stages] | empty[stages] | chunk_full[2] | chunk_free[2] | done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * P::STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + P::STAGES + s); };
  auto chunk_full = [&](int b) { return smem_u32(bars + 2 * P::STAGES + b); };
  auto chunk_free = [&](int b) { return smem_u32(bars + 2 * P::STAGES + 2 + b); };
  const uint32_t done_bar = smem_u32(bars + 2 * P::STAGES + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int2 tile = tiles[blockIdx.x];
  const int p0 = tile.x * DBM, q0 = tile.y * DBN;
  const int nchunks = (nk + CHUNK_STAGES - 1) / CHUNK_STAGES;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P::STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(chunk_full(b), 1);
      mbar_init(chunk_free(b), 8);  // one arrival per epilogue warp
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
        const int s = kb % P::STAGES;
        const uint32_t ph = (uint32_t)(kb / P::STAGES) & 1u;
        if (!mbar_wait(empty(s), ph ^ 1u, abort_flag)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t dst = sbase + s * P::STAGE_BYTES;
        mbar_expect_tx(full(s), P::STAGE_BYTES);
        tma_load_3d(dst, &tmA, kb * DSK, p0, 0, full(s));
        tma_load_3d(dst + P::NA * A_PLANE, &tmB, kb * DSK, q0, 0, full(s));
        issued = kb + 1;
      }
      if (*abort_flag) {  // let every issued copy land before the CTA can exit
        for (int kb = issued > P::STAGES ? issued - P::STAGES : 0; kb < issued; ++kb)
          mbar_wait(full(kb % P::STAGES), (uint32_t)(kb / P::STAGES) & 1u, nullptr);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      for (int kb = 0; kb < nk && !*abort_flag; ++kb) {
        const int c = kb / CHUNK_STAGES, buf = c & 1;
        const bool chunk_start = (kb % CHUNK_STAGES) == 0;
        if (chunk_start && c >= 2 &&
            !mbar_wait(chunk_free(buf), (uint32_t)((c >> 1) - 1) & 1u, abort_flag)) {
          *abort_flag = 1;
          break;
        }
        const int s = kb % P::STAGES;
        if (!mbar_wait(full(s), (uint32_t)(kb / P::STAGES) & 1u, abort_flag)) {
          *abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t stage = sbase + s * P::STAGE_BYTES;
        const uint32_t dbuf = tmem + (uint32_t)buf * BUF_COLS;
#pragma unroll
        for (int da = 0; da < P::NA; ++da) {
          // the pairs (da, t) of the pass have consecutive t; their B planes
          // lie one after another in the stage (64 rows each, the same 8-row
          // group stride) and their weights' accumulators one after another
          // in tensor memory, so one MMA with N = 64 x (pairs) covers them
          const int t0 = P::first_t(da), t1 = P::last_t(da);
          if (t1 < t0) continue;
          const uint64_t ad = sdesc_sw64(stage + da * A_PLANE);
          const uint64_t bd = sdesc_sw64(stage + P::NA * A_PLANE + t0 * B_PLANE);
          const uint32_t d = dbuf + (uint32_t)((da + t0 - P::W0) * DBN);
          const uint32_t idesc = idesc_bf16(DBM, DBN * (t1 - t0 + 1));
#pragma unroll
          for (int k = 0; k < DSK / 16; ++k) {  // 32 bytes (16 BF16) along K per MMA
            // the MMA of A digit 0 covers every weight of the pass: at the
            // chunk's first K step it starts all of their accumulators
            const uint32_t accum = (chunk_start && da == 0 && k == 0) ? 0u : 1u;
            umma_f16(d, ad + 2 * k, bd + 2 * k, idesc, accum);
          }
        }
        umma_commit(empty(s));
        if ((kb % CHUNK_STAGES) == CHUNK_STAGES - 1 || kb == nk - 1) umma_commit(chunk_full(buf));
      }
      umma_commit(done_bar);  // fires once every MMA issued above has completed
      mbar_wait(done_bar, 0, nullptr);
    }
    __syncwarp();
  } else {
    const int quarter = warp & 3;         // TMEM lanes this warp may read
    const int half = (warp - 2) >> 2;     // its 32 columns of each weight block
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 32);
    // exact integer sums of this lane's row, 32 columns: sum over the pass's
    // weights of I_w 2^(8(3 - (w - W0))) (|I_w| < 2^24 per chunk and at most
    // 5 2^14 k <= 5 2^28 over all columns: the int64 sums stay below 2^55)
    long long acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0;
    int ok = 1;
    for (int c = 0; c < nchunks; ++c) {
      const int buf = c & 1;
      if (lane == 0) ok = mbar_wait(chunk_full(buf), (uint32_t)(c >> 1) & 1u, abort_flag) && !*abort_flag;
      ok = __shfl_sync(0xffffffffu, ok, 0);  // warp-uniform for tcgen05.ld
      if (!ok) break;
      fence_after();
#pragma unroll
      for (int wl = 0; wl < NWP; ++wl) {
        uint32_t r[32];
        tmem_ld32(lane_addr + (uint32_t)buf * BUF_COLS + (uint32_t)(wl * DBN), r);
#pragma unroll
        for (int j = 0; j < 32; ++j)
          acc[j] += (long long)__float2int_rn(__uint_as_float(r[j])) * (1ll << (8 * (NWP - 1 - wl)));
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(chunk_free(buf));
    }
    if (ok) {
      const int64_t p = p0 + quarter * 32 + lane;
      if (p < m) {
        long long* dst = reinterpret_cast<long long*>(M + p * ldm);
        const int64_t qb = (int64_t)q0 + half * 32;
        if (PASS == 0) {  // hi, as int64 bits, until pass 1
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            const int64_t q = qb + j;
            if (q + 1 <= p) *reinterpret_cast<longlong2*>(dst + q) = make_longlong2(acc[j], acc[j + 1]);
            else if (q <= p) dst[q] = acc[j];
          }
        } else {
          const int ep = ea[p];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int64_t q = qb + j;
            // sum_w 2^(-8w) I_w = 2^-24 (hi + 2^-32 lo), two FP64 roundings
            if (q <= p) {
              const long long hi = dst[q];
              M[p * ldm + q] = ldexp(fma((double)acc[j], 0x1p-32, (double)hi), ep + eb[q] - 38);
            }
          }
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

// The prepass reads BF16 A and FP64 D as bit fields, on the integer pipes
// (GB300 runs FP64 at 1/64 of the FP32 rate): a finite value is sig 2^e with
// an integer significand sig (the implicit one included, subnormals as they
// are).  A_pj D_j is then the exact integer product sig_a sig_d (at most
// 8 + 53 bits) times 2^(e_a + e_d).
__device__ __forceinline__ void bf16_fields(uint16_t h, unsigned long long& sig, int& e) {
  const int E = (h >> 7) & 0xff;
  sig = (unsigned long long)((h & 0x7fu) | (E ? 0x80u : 0u));
  e = (E ? E : 1) - 127 - 7;
}
__device__ __forceinline__ void f64_fields(unsigned long long bits, unsigned long long& sig, int& e) {
  const int E = (int)((bits >> 52) & 0x7ff);
  sig = (bits & 0xfffffffffffffull) | (E ? (1ull << 52) : 0ull);
  e = (E ? E : 1) - 1023 - 52;
}
// frexp exponent of sig 2^e, sig > 0: the bit length of sig plus e.
__device__ __forceinline__ int frexp_exp(unsigned long long sig, int e) { return 64 - __clzll((long long)sig) + e; }

// Exponents of the kept part of each row: ea_p with max_j |A_pj| < 2^ea_p and
// eb_p with max_j |D_j A_pj| < 2^eb_p (frexp convention; 0 for a zero row),
// eb_p from the exact products.  One warp per row; column i of the kept set
// is idx[i] (idx null: i).  D > 0.
__global__ void k_dig_rowexp(int64_t m, int64_t n, const __nv_bfloat16* __restrict__ A, const double* __restrict__ D,
                             int64_t k, const int* __restrict__ idx, int* __restrict__ ea, int* __restrict__ eb) {
  const int lane = threadIdx.x & 31;
  const uint16_t* Ab = reinterpret_cast<const uint16_t*>(A);
  const unsigned long long* Db = reinterpret_cast<const unsigned long long*>(D);
  for (int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; p < m;
       p += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const uint16_t* row = Ab + p * n;
    unsigned amag = 0;   // largest |A_pj| as BF16 magnitude bits (ordered like the values)
    int ebm = INT_MIN;   // largest frexp exponent of A_pj D_j
    constexpr int U = 8;  // gathers in flight per lane
    for (int64_t i0 = lane; i0 < k; i0 += 32 * U) {
      int64_t j[U];
      uint16_t h[U];
      unsigned long long dbits[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + 32 * u;
        j[u] = i < k ? (idx ? (int64_t)idx[i] : i) : -1;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        h[u] = j[u] >= 0 ? row[j[u]] : (uint16_t)0;
        dbits[u] = j[u] >= 0 ? __ldg(Db + j[u]) : 0ull;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const unsigned mag = h[u] & 0x7fffu;
        if (mag == 0) continue;
        amag = max(amag, mag);
        unsigned long long sa, sd;
        int e_a, e_d;
        bf16_fields(h[u], sa, e_a);
        f64_fields(dbits[u], sd, e_d);
        ebm = max(ebm, frexp_exp(sa * sd, e_a + e_d));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      amag = max(amag, __shfl_xor_sync(0xffffffffu, amag, o));
      ebm = max(ebm, __shfl_xor_sync(0xffffffffu, ebm, o));
    }
    if (lane == 0) {
      int e1 = 0;
      if (amag) {
        unsigned long long sa;
        int e_a;
        bf16_fields((uint16_t)amag, sa, e_a);
        e1 = frexp_exp(sa, e_a);
      }
      ea[p] = e1;
      eb[p] = ebm == INT_MIN ? 0 : ebm;
    }
  }
}

// v 2^s rounded to the nearest integer (ties to even), v >= 0; for s >= 0 the
// caller keeps v 2^s below 2^63.
__device__ __forceinline__ unsigned long long shift_rne(unsigned long long v, int s) {
  if (s >= 0) return v << s;
  const int r = -s;
  if (r >= 64) return 0ull;  // v < 2^61: below half of 2^r
  const unsigned long long q = v >> r, rem = v & ((1ull << r) - 1ull), half = 1ull << (r - 1);
  return q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
}

// Balanced base-256 digits of the integer v (|v| < 2^(8 ND - 1) + 2^7):
// dig[ND - 1] is the lowest; each in [-128, 128].
template <int ND>
__device__ __forceinline__ void balanced_digits(long long v, int (&dig)[ND]) {
#pragma unroll
  for (int t = ND - 1; t > 0; --t) {
    const int low = (int)(((v + 128) & 255) - 128);
    dig[t] = low;
    v = (v - low) >> 8;  // exact: v - low is a multiple of 256
  }
  dig[0] = (int)v;
}

__device__ __forceinline__ uint32_t bf16_pair(int lo, int hi) {
  return bf16_bits_small(lo) | (bf16_bits_small(hi) << 16);
}

// The digit planes: plane s of A (SA planes) and plane t of B (SB planes),
// each mpad rows of stride kstride BF16, for the kept columns i < k (and
// zeros up to the next multiple of 64).  a' = A_pj 2^(39 - ea_p) and
// b' = A_pj D_j 2^(63 - eb_p) rounded to integers (exact except for entries
// below 2^-32 of the row's largest in a' and for the bits of the exact
// product below 2^-63 of 2^eb_p in b'), both on the integer pipes; their
// balanced base-256 digits are the planes' entries.  One thread writes 8
// consecutive columns of one row to every plane.
__global__ void k_dig_planes(int64_t m, int64_t n, const __nv_bfloat16* __restrict__ A, const double* __restrict__ D,
                             int64_t k, int64_t kfill, const int* __restrict__ idx, const int* __restrict__ ea,
                             const int* __restrict__ eb, int64_t mpad, int64_t kstride,
                             __nv_bfloat16* __restrict__ planes) {
  const int64_t groups = kfill / 8;
  const int64_t total = m * groups;
  const int64_t plane = mpad * kstride;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = g / groups, i0 = (g % groups) * 8;
    const int sha = 39 - ea[p], shb = 63 - eb[p];
    int da[8][SA], db[8][SB];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int64_t i = i0 + e;
      long long av = 0, bv = 0;
      if (i < k) {
        const int64_t j = idx ? idx[i] : i;
        const uint16_t h = reinterpret_cast<const uint16_t*>(A)[p * n + j];
        unsigned long long sa, sd;
        int e_a, e_d;
        bf16_fields(h, sa, e_a);
        f64_fields(__ldg(reinterpret_cast<const unsigned long long*>(D) + j), sd, e_d);
        av = (long long)shift_rne(sa, e_a + sha);
        bv = (long long)shift_rne(sa * sd, e_a + e_d + shb);
        if (h & 0x8000u) {
          av = -av;
          bv = -bv;
        }
      }
      balanced_digits<SA>(av, da[e]);
      balanced_digits<SB>(bv, db[e]);
    }
    __nv_bfloat16* rowp = planes + p * kstride + i0;
#pragma unroll
    for (int s = 0; s < SA; ++s)
      *reinterpret_cast<uint4*>(rowp + s * plane) = make_uint4(bf16_pair(da[0][s], da[1][s]), bf16_pair(da[2][s], da[3][s]),
                                                               bf16_pair(da[4][s], da[5][s]), bf16_pair(da[6][s], da[7][s]));
#pragma unroll
    for (int t = 0; t < SB; ++t)
      *reinterpret_cast<uint4*>(rowp + (SA + t) * plane) =
          make_uint4(bf16_pair(db[0][t], db[1][t]), bf16_pair(db[2][t], db[3][t]), bf16_pair(db[4][t], db[5][t]),
                     bf16_pair(db[6][t], db[7][t]));
  }
}

// ---- host side ---------------------------------------------------------------
struct DigHost {
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  CUtensorMap mapA[2], mapB[2];  // per pass: A digits 0-3 / 0-4, B digits 0-3 / 0-7
  int2* tiles = nullptr;
  int ntiles = 0;
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

// 3-D BF16 map over `planes` consecutive digit planes: dims {kstride (K,
// innermost), mpad, planes}, box {32 (one 64-byte row), rows, box_planes},
// 64-byte swizzle.  The box lands in shared memory as box_planes x rows x
// 64 B.
cudaError_t encode_planes(DigHost* hs, CUtensorMap* map, const void* base, int64_t mpad, int64_t kstride, int planes,
                          int box_planes, int rows) {
  cuuint64_t dims[3] = {(cuuint64_t)kstride, (cuuint64_t)mpad, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(kstride * 2), (cuuint64_t)(mpad * kstride * 2)};
  cuuint32_t box[3] = {(cuuint32_t)DSK, (cuuint32_t)rows, (cuuint32_t)box_planes};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = hs->encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t dig_workspace_create(DigWorkspace* w, int64_t m, int64_t n) {
  w->m = m;
  w->mpad = (m + DBM - 1) / DBM * DBM;
  const int64_t kmax = std::min<int64_t>(n, kDigMaxK);
  w->kstride = (kmax + DBK - 1) / DBK * DBK;
  DigHost* hs = new (std::nothrow) DigHost();
  if (!hs) return cudaErrorMemoryAllocation;
  w->host = hs;
  cudaError_t e = get_encoder(&hs->encode);
  if (e == cudaSuccess) e = cudaMalloc(&w->planes, sizeof(__nv_bfloat16) * (size_t)(SA + SB) * w->mpad * w->kstride);
  // zero once: rows m..mpad of every plane are never written and must read as 0
  if (e == cudaSuccess) e = cudaMemset(w->planes, 0, sizeof(__nv_bfloat16) * (size_t)(SA + SB) * w->mpad * w->kstride);
  if (e == cudaSuccess) e = cudaMalloc(&w->ea, sizeof(int) * (size_t)m);
  if (e == cudaSuccess) e = cudaMalloc(&w->eb, sizeof(int) * (size_t)w->mpad);
  if (e == cudaSuccess) e = cudaMemset(w->eb, 0, sizeof(int) * (size_t)w->mpad);
  // Lower-triangle tiles (I, J) of 128 x 64 (some row p >= some column q),
  // in super-tiles of G row blocks x 2G column blocks, so the CTAs resident
  // together share their digit planes in L2.
  std::vector<int2> tl;
  const int64_t nI = w->mpad / DBM, nJ = (m + DBN - 1) / DBN;
  const int64_t G = 6;
  for (int64_t PI = 0; PI < nI; PI += G)
    for (int64_t PJ = 0; PJ < nJ; PJ += 2 * G)
      for (int64_t I = PI; I < nI && I < PI + G; ++I)
        for (int64_t J = PJ; J < nJ && J < PJ + 2 * G && J * DBN <= I * DBM + DBM - 1; ++J)
          tl.push_back(make_int2((int)I, (int)J));
  hs->ntiles = (int)tl.size();
  if (e == cudaSuccess) e = cudaMalloc(&hs->tiles, sizeof(int2) * tl.size());
  if (e == cudaSuccess) e = cudaMemcpy(hs->tiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice);
  const void* bplanes = (const __nv_bfloat16*)w->planes + (size_t)SA * w->mpad * w->kstride;
  if (e == cudaSuccess) e = encode_planes(hs, &hs->mapA[0], w->planes, w->mpad, w->kstride, SA, DigPass<0>::NA, DBM);
  if (e == cudaSuccess) e = encode_planes(hs, &hs->mapA[1], w->planes, w->mpad, w->kstride, SA, DigPass<1>::NA, DBM);
  if (e == cudaSuccess) e = encode_planes(hs, &hs->mapB[0], bplanes, w->mpad, w->kstride, SB, DigPass<0>::NB, DBN);
  if (e == cudaSuccess) e = encode_planes(hs, &hs->mapB[1], bplanes, w->mpad, w->kstride, SB, DigPass<1>::NB, DBN);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_syrk_dig<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DigPass<0>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_syrk_dig<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DigPass<1>::SMEM_BYTES);
  return e;
}

void dig_workspace_destroy(DigWorkspace* w) {
  if (w->planes) cudaFree(w->planes);
  if (w->ea) cudaFree(w->ea);
  if (w->eb) cudaFree(w->eb);
  DigHost* hs = static_cast<DigHost*>(w->host);
  if (hs) {
    if (hs->tiles) cudaFree(hs->tiles);
    delete hs;
  }
  *w = DigWorkspace{};
}

cudaError_t dig_syrk(cudaStream_t st, DigWorkspace* w, const __nv_bfloat16* A, int64_t n, const double* D, int64_t k,
                     const int* idx, double* M64, int64_t ldm, Scalars* sc, int* launches) {
  *launches = 0;
  if (k < 1 || k > w->kstride || w->m < 1) return cudaErrorInvalidValue;
  DigHost* hs = static_cast<DigHost*>(w->host);
  const int64_t m = w->m;
  const int64_t kfill = (k + DBK - 1) / DBK * DBK;  // the stages read columns < kfill
  {
    const int64_t warps = m, threads = warps * 32;
    const unsigned grid = (unsigned)std::min<int64_t>((threads + 255) / 256, 4736);
    k_dig_rowexp<<<grid, 256, 0, st>>>(m, n, A, D, k, idx, w->ea, w->eb);
  }
  {
    const int64_t work = m * (kfill / 8);
    const unsigned grid = (unsigned)std::min<int64_t>((work + 255) / 256, 4736);
    k_dig_planes<<<grid, 256, 0, st>>>(m, n, A, D, k, kfill, idx, w->ea, w->eb, w->mpad, w->kstride,
                                       static_cast<__nv_bfloat16*>(w->planes));
  }
  const int nk = (int)(kfill / DSK);
  k_syrk_dig<0><<<(unsigned)hs->ntiles, NUM_THREADS, DigPass<0>::SMEM_BYTES, st>>>(
      hs->mapA[0], hs->mapB[0], hs->tiles, nk, m, w->ea, w->eb, ldm, M64, sc);
  k_syrk_dig<1><<<(unsigned)hs->ntiles, NUM_THREADS, DigPass<1>::SMEM_BYTES, st>>>(
      hs->mapA[1], hs->mapB[1], hs->tiles, nk, m, w->ea, w->eb, ldm, M64, sc);
  *launches = 4;
  return cudaGetLastError();
}

}  // namespace pdas
