// chol_dig.cu -- FP64 blocked Cholesky of the FP64 tier (Section V-A's
// symmetric positive definite solve) whose trailing updates run on the
// tcgen05 tensor cores, exactly, from fixed-point BF16 digit planes.
//
// Per 64-column panel k0 (kb = min(64, m - k0) columns):
//   k_dig_diag                      -- the FP64 factor L_11 of the diagonal
//                                      block (LDL' form) and 1 / L_cc: a
//                                      launch of its own for the first panel;
//                                      for the others CTA 0 of the previous
//                                      panel's update factors the block right
//                                      after writing tiles 0 and 1, which
//                                      hold it, while the other CTAs update
//                                      the rest;
//   k_dig_panel_rows                -- the panel rows P (trailing rows
//                                      r >= k0 + kb, the kb panel columns)
//                                      solved in FP64, P L_11' = B, 32 rows
//                                      per CTA over every SM; each row then
//                                      written as 7 balanced base-256 digits
//                                      of P_rc 2^-e_r, e_r the exponent of
//                                      the row's largest |P_rc|:
//                                      P_rc = 2^e_r sum_s d_s 2^(-7-8s);
//   k_dig_update                    -- C_pq -= (P P')_pq over the lower tiles
//                                      (128 rows p x 32 columns q) of the
//                                      trailing matrix:
//        (P P')_pq = 2^(e_p + e_q - 14) sum_{w<=7} 2^(-8w) I_w,
//        I_w = sum_c sum_{s+t=w} d_s,pc d_t,qc,
//      every digit product an integer of magnitude <= 2^14, at most 7 pairs
//      per weight and kb <= 64 columns: |I_w| < 2^23, so the tensor core's
//      FP32 accumulator holds I_w exactly.  The epilogue combines the eight
//      weights into one int64 (the last two rounded to 2^-43 of the sum),
//      builds the double on the integer pipes and subtracts it from C in
//      FP64.
// The only roundings of an update are the digits of entries below 1/8 of
// their row's largest (to 2^-56 of 2^e_r), the digit pairs of weight 8 and
// more left out (at most 2^-62 of 2^(e_p + e_q) per column), the rounding of
// the two lowest weights (2^-57 of 2^(e_p + e_q)), the conversion to FP64 and
// the subtraction: FP64-grade, where the FP64 pipes would take 1/64 of the
// FP32 rate.
//
// k_dig_update: persistent, one CTA per SM over a contiguous range of the
// 128 x 32 tiles, 18 warps, two tiles in flight:
//   warp 0      TMA: the 7 planes of the tile's rows p (128 x 64 columns,
//               112 KB) once per row block, and per tile the 7 planes of its
//               rows q (32 x 64 columns, 28 KB) into one of two buffers;
//   warp 1      allocates 512 TMEM columns (2 buffers x 8 weights x 32); one
//               lane issues tcgen05.mma.cta_group::1.kind::f16 (M = 128,
//               N = 32 x pairs, K = 16): 8 groups of the 34 digit pairs x 4
//               K steps, pair (s, t) into weight s + t, as soon as the tile's
//               planes have landed and the epilogue has read the buffer's
//               previous tile;
//   warps 2..17 thread (warp w, lane) owns row 32 (w % 4) + lane of the tile
//               and columns 8 ((w - 2) / 4).. of it: it reads its TMEM lane
//               of every weight, combines the weights into one integer per
//               entry and releases the buffer; the scaled updates then go
//               through a per-warp staging area, and C is read (before the
//               MMA wait) and written back in a coalesced layout.
// Every mbarrier wait is bounded (2 s); on a timeout the CTA sets
// PDAS_ERR_TIMEOUT, lets its copy land and its MMAs finish, frees TMEM, exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "chol_dig.cuh"
#include "tc_util.cuh"

namespace pdas {

namespace {

using namespace tc;

constexpr int UBM = 128;                          // rows p of a tile
constexpr int UBN = 32;                           // rows q (columns of C) of a tile
constexpr int UK = 64;                            // panel width (columns of P): one 128-byte row
constexpr int ND = 7;                             // digits per entry (55 bits)
constexpr int WMAX = 7;                           // largest pair weight kept
constexpr int NW = WMAX + 1;
constexpr int NPAIR = 34;                         // pairs (s, t), s, t < 7, s + t <= 7
static_assert(NPAIR == 7 + 7 + 6 + 5 + 4 + 3 + 2, "pair count");
constexpr uint32_t P_PLANE = UBM * 128;           // 16 KB: 128 rows of one digit
constexpr uint32_t Q_PLANE = UBN * 128;           // 4 KB: 32 rows of one digit
constexpr uint32_t P_BYTES = ND * P_PLANE;        // 112 KB: the P planes of a row block of tiles
constexpr uint32_t Q_BYTES = ND * Q_PLANE;        // 28 KB: the Q planes of a tile (two buffers)
constexpr uint32_t LOAD_BYTES = P_BYTES + 2 * Q_BYTES;  // 168 KB
constexpr uint32_t BUF_COLS = NW * UBN;           // 256: the 8 weight accumulators of a tile
constexpr uint32_t TMEM_COLS = 2 * BUF_COLS;      // 512: two tiles in flight
constexpr int NUM_THREADS = 576;                  // 2 role warps + 16 epilogue warps
constexpr int EPI_WARPS = NUM_THREADS / 32 - 2;
// Per epilogue warp, a 32-row staging area for the scaled updates (8 columns,
// pitch 9 doubles): C is read and written in a coalesced layout while the
// updates are formed with one tile row per lane (the tensor-memory layout).
constexpr int STG_PITCH = 9;
constexpr size_t STG_BYTES = (size_t)(NUM_THREADS / 32 - 2) * 32 * STG_PITCH * sizeof(double);
constexpr size_t SMEM_BYTES = 1024 + (size_t)LOAD_BYTES + 256 + STG_BYTES;

// The pairs (s, t) with a fixed s have consecutive t; the Q planes t lie one
// after another in shared memory (32 rows each, the same 8-row group stride)
// and the accumulators of the weights s + t one after another in tensor
// memory, so one MMA with N = 32 x (pairs) covers them.  A group starts its
// weights' accumulators (no accumulation at its first K step) when it holds
// the first product of each of them: pair (0, w), or (1, 6) for w = 7, which
// therefore gets a group of its own.
struct MmaGroup {
  int s, t0, nt;
  bool first;
};
constexpr int NGROUP = 8;
__host__ __device__ constexpr MmaGroup mma_group(int g) {
  constexpr MmaGroup G[NGROUP] = {{0, 0, 7, true},  {1, 0, 6, false}, {1, 6, 1, true},  {2, 0, 6, false},
                                  {3, 0, 5, false}, {4, 0, 4, false}, {5, 0, 3, false}, {6, 0, 2, false}};
  return G[g];
}
// the groups cover each pair (s, t), s + t <= WMAX, once; a group's first
// flag holds exactly when each of its weights first appears in it
constexpr bool groups_ok() {
  int seen[ND][ND] = {};
  bool started[NW] = {};
  int pairs = 0;
  for (int g = 0; g < NGROUP; ++g) {
    const MmaGroup G = mma_group(g);
    if (G.nt < 1 || UBN * G.nt > 256 || G.t0 + G.nt > ND) return false;
    for (int t = G.t0; t < G.t0 + G.nt; ++t) {
      if (G.s + t > WMAX || seen[G.s][t]++) return false;
      if (started[G.s + t] == G.first) return false;
      ++pairs;
    }
    for (int t = G.t0; t < G.t0 + G.nt; ++t) started[G.s + t] = true;
  }
  return pairs == NPAIR;
}
static_assert(groups_ok(), "MMA groups of the digit pairs");

static_assert(SMEM_BYTES <= 232448, "shared memory of one CTA");

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* map, int c0, int c1, int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// z 2^k as a double, rounded to nearest (ties to even), built on the
// integer pipes: the leading one of |z| found by a count of leading zeros,
// the 53-bit significand shifted out and rounded, the exponent field set to
// the position of the leading one plus k.  Subnormal and overflowing
// results take the FP64 path.
__device__ __forceinline__ double scaled_int_to_double(long long z, int k) {
  if (z == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)z & 0x8000000000000000ull;
  const unsigned long long a = z < 0 ? 0ull - (unsigned long long)z : (unsigned long long)z;
  const int lz = __clzll((long long)a);
  const unsigned long long nrm = a << lz;  // leading one at bit 63
  unsigned long long mant = nrm >> 11;     // leading one at bit 52
  const unsigned rest = (unsigned)nrm & 0x7ffu;
  mant += (rest > 0x400u || (rest == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
  const int ex = 1023 + 63 - lz + k;  // biased exponent of |z| 2^k
  if (ex <= 0 || ex >= 2046) return ldexp((double)z, k);
  // the leading one of mant adds 1 to the field (2 when the rounding carried
  // into bit 53, which is then the right exponent with a zero fraction)
  return __longlong_as_double((long long)(sgn | (((unsigned long long)(ex - 1) << 52) + mant)));
}

// Balanced base-256 digits of the integer v: dig[ND - 1] the lowest, each in
// [-128, 128].
__device__ __forceinline__ void balanced_digits(long long v, int (&dig)[ND]) {
#pragma unroll
  for (int t = ND - 1; t > 0; --t) {
    const int low = (int)(((v + 128) & 255) - 128);
    dig[t] = low;
    v = (v - low) >> 8;
  }
  dig[0] = (int)v;
}

// GB300's FP64 pipes take ~64 cycles per warp instruction per SM
// sub-partition, whatever the number of active lanes, and ~64 cycles of
// latency per dependent operation (a reciprocal ~430).  The two FP64 kernels
// of the panel are laid out for that: every FP64 instruction they issue has
// (nearly) all its lanes busy, and the chain from one column to the next is
// a handful of dependent operations.

// 1 / d of a pivot d, or -1 when d is not positive and finite or its
// reciprocal overflows.
__device__ __forceinline__ double inv_pivot(double d) {
  const double r = __drcp_rn(d);
  return (d > 0.0 && isfinite(d) && isfinite(r)) ? r : -1.0;
}

// The FP64 factor of the kb x kb diagonal block of panel k0 (kb <= 64) by one
// CTA, right-looking in the LDL' form (an identity past kb), one barrier per
// column.  At step c the first warp (the "pivot warp", lane l holding rows l
// and l + 32) finishes column c + 1: M_i,c+1 -= t_ic M_c+1,c for its rows,
// the pivot d_c+1 (row c + 1), 1 / d_c+1, and t_i,c+1 = M_i,c+1 / d_c+1, and
// posts t and M of column c + 1.  Meanwhile the "bulk" warps apply column c
// to the columns past c + 1, M_ij -= t_ic M_jc, and post column c + 2.
// GB300's FP64 pipe runs one warp instruction per ~64 cycles per SM
// sub-partition, whatever the number of active lanes, so:
//   - the bulk's entries are ordered by column from the last to the first
//     (rows ascending inside a column) and dealt to its threads in turn,
//     entry (i, j), i >= j, at e = P(j) + i - j, P(j) = (63 - j)(64 - j) / 2:
//     the entries of the columns past c + 1 are the first P(c + 1), so every
//     FP64 instruction has all lanes busy but the last, and column c + 2,
//     posted next, comes last in the order (a thread updates its slots from
//     the highest down);
//   - the warps on the pivot warp's sub-partition take no bulk entries, so
//     the dependent chain of the pivot (a multiply-add, the reciprocal, a
//     multiply per column) never queues behind the bulk.
// Each entry receives the same operations in the same order as in a sweep
// over the trailing triangle.  The square roots and the scaling
// L_ic = M_ic / sqrt(d_c) then run for all columns at once.  Writes L_11
// (lower triangle and diagonal) to M and 1 / L_cc to dinv[k0 + c]; a pivot
// that is not positive and finite sets PDAS_ERR_NOT_SPD with its index.
constexpr int DG_THREADS = 256;
struct DiagSmem {
  double Ld[UK][UK + 1];  // the block, staged (coalesced loads and stores); then M_ic of finished columns
  double w[2][UK];        // column c + 2 from the bulk (alternating halves)
  double t[2][UK];        // t_ic of column c (alternating halves)
  double u[2][UK];        // M_ic of column c (alternating halves)
  double dg[UK];          // the pivots d_c
  double s_rp[UK];        // 1 / L_cc
  int fail;               // first column whose pivot failed, or -1
};
__host__ __device__ constexpr int diag_col_start(int j) { return (UK - 1 - j) * (UK - j) / 2; }

// The factor itself, by NT threads (tid; warp w = tid / 32 runs on SM
// sub-partition w mod 4 up to a common offset) that meet at bar().
template <int NT, class Bar>
__device__ __forceinline__ void diag_factor(int64_t ldm, double* __restrict__ M, double* __restrict__ dinv,
                                            int64_t k0, int kb, Scalars* sc, DiagSmem& S, int tid, Bar bar) {
  constexpr int NBULK = NT / 4 * 3;                     // threads of the bulk warps
  constexpr int NS = (diag_col_start(1) + NBULK - 1) / NBULK;  // slots: the columns past 1 at most
  const int wq = tid >> 5, lane = tid & 31;
  const bool pivot_warp = wq == 0, bulk = (wq & 3) != 0;
  const int b = (wq - (wq >> 2) - 1) * 32 + lane;       // bulk index
  for (int t = tid; t < UK * UK; t += NT) {
    const int i = t / UK, j = t % UK;
    if (j <= i) S.Ld[i][j] = i < kb ? M[(k0 + i) * ldm + k0 + j] : (i == j ? 1.0 : 0.0);
  }
  if (tid == 0) S.fail = -1;
  bar();
  double v[NS];
  int ij[NS];  // i << 8 | j of the slot's entry
  if (bulk) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int e = b + s * NBULK;
      int i = UK - 1, j = UK - 1;  // (a slot past the columns it serves: never updated, never posted)
      if (e < diag_col_start(1)) {
        int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);  // FP32 estimate, corrected below
        while (r * (r + 1) / 2 > e) --r;
        while ((r + 1) * (r + 2) / 2 <= e) ++r;
        j = UK - 1 - r;  // diag_col_start(j) = r (r + 1) / 2
        i = j + (e - r * (r + 1) / 2);
      }
      ij[s] = (i << 8) | j;
      v[s] = S.Ld[i][j];
    }
  }
  if (tid < UK) S.w[1][tid] = S.Ld[tid][1];  // column 1 before any update
  // pivot warp: column 0 (t and M of its rows lane, lane + 32 in registers)
  double t0 = 0.0, t1 = 0.0, u0 = 0.0, u1 = 0.0;
  if (pivot_warp) {
    u0 = S.Ld[lane][0];
    u1 = S.Ld[lane + 32][0];
    const double d = S.Ld[0][0], inv = inv_pivot(d);
    t0 = u0 * inv;
    t1 = u1 * inv;
    S.t[0][lane] = t0;
    S.t[0][lane + 32] = t1;
    S.u[0][lane] = u0;
    S.u[0][lane + 32] = u1;
    if (lane == 0) {
      S.dg[0] = d;
      if (inv < 0.0) S.fail = 0;
    }
  }
  bar();
  int fail = S.fail;
  for (int c = 0; c + 1 < kb && fail < 0; ++c) {
    if (pivot_warp) {
      const double* wb = S.w[(c + 1) & 1];
      const double w0 = wb[lane], w1 = wb[lane + 32];
      const int pr = (c + 1) & 31;
      const bool hi = c + 1 >= 32;
      const double up = __shfl_sync(0xffffffffu, hi ? u1 : u0, pr);  // M_c+1,c
      const double n0 = fma(-t0, up, w0), n1 = fma(-t1, up, w1);     // M_i,c+1
      const double d = __shfl_sync(0xffffffffu, hi ? n1 : n0, pr);   // d_c+1
      const double inv = inv_pivot(d);
      t0 = n0 * inv;
      t1 = n1 * inv;
      u0 = n0;
      u1 = n1;
      double* tb = S.t[(c + 1) & 1];
      double* ub = S.u[(c + 1) & 1];
      tb[lane] = t0;
      tb[lane + 32] = t1;
      ub[lane] = u0;
      ub[lane + 32] = u1;
      if (lane > c + 1) S.Ld[lane][c + 1] = u0;
      if (lane + 32 > c + 1) S.Ld[lane + 32][c + 1] = u1;
      if (lane == 0) {
        S.dg[c + 1] = d;
        if (inv < 0.0) S.fail = c + 1;
      }
    } else if (bulk) {
      const double* tc = S.t[c & 1];
      const double* uc = S.u[c & 1];
      double* wn = S.w[c & 1];  // column c + 2 (buffer (c + 2) & 1)
      const int ne = diag_col_start(c + 1), ne2 = diag_col_start(c + 2);
#pragma unroll
      for (int s = NS - 1; s >= 0; --s) {
        const int e = b + s * NBULK;
        if (e < ne) {
          const int i = ij[s] >> 8, j = ij[s] & 0xff;
          v[s] = fma(-tc[i], uc[j], v[s]);
          if (e >= ne2) wn[i] = v[s];  // column c + 2, all of its updates up to column c applied
        }
      }
    }
    bar();
    fail = S.fail;
  }
  if (fail >= 0) {  // every thread read the same index
    if (tid == 0 && atomicCAS(&sc->status, 0, (int)PDAS_ERR_NOT_SPD) == 0) sc->fail_index = (int)(k0 + fail);
    return;
  }
  if (tid < kb) {
    const double l = sqrt(S.dg[tid]);
    S.Ld[tid][tid] = l;
    S.s_rp[tid] = 1.0 / l;
    dinv[k0 + tid] = S.s_rp[tid];
  }
  bar();
  for (int t = tid; t < UK * UK; t += NT) {
    const int i = t / UK, j = t % UK;
    if (j <= i && i < kb) M[(k0 + i) * ldm + k0 + j] = j < i ? S.Ld[i][j] * S.s_rp[j] : S.Ld[i][i];
  }
}

// The first panel's diagonal block (the others are factored inside the
// previous panel's update, k_dig_update).
__global__ void __launch_bounds__(DG_THREADS) k_dig_diag(int64_t ldm, double* __restrict__ M,
                                                         double* __restrict__ dinv, int64_t k0, int kb, Scalars* sc) {
  __shared__ DiagSmem S;
  if (*(volatile const int*)&sc->status != 0) return;
  diag_factor<DG_THREADS>(ldm, M, dinv, k0, kb, sc, S, (int)threadIdx.x, [] { __syncthreads(); });
}

// The panel rows r = k0 + kb + i (i < rows): X L_11' = B in FP64 (B the kb
// panel columns of the rows, L_11 and 1 / L_cc from the diagonal factor),
// X written back to M; then the digits of X into planes (7 planes of mpad
// rows x 64 columns, BF16) and the row exponents into e[i].
// Solve: T threads per row; thread `part` of a row holds columns part,
// part + T, ... in registers.  The sweep over the columns is unrolled at
// compile time, so at column c a thread issues multiply-adds only for its
// slots that can still lie past c (at most one of them predicated off):
// column c's value x_c = b_c / L_cc is formed by its owner and passed to
// the row's other threads by a shuffle.  Small T gives the fewest FP64
// instructions per row, large T the shortest sweep per warp; the host picks
// T per panel from the number of rows.  Digits: one warp per row, the lanes
// holding columns 2 lane and 2 lane + 1 (whole 128-byte plane rows).
constexpr int PR_THREADS = 128;

template <int T>
__global__ void __launch_bounds__(PR_THREADS) k_dig_panel_rows(int64_t ldm, double* __restrict__ M,
                                                             const double* __restrict__ dinv, int64_t k0, int kb,
                                                             int64_t rows, int64_t mpad, int* __restrict__ e,
                                                             __nv_bfloat16* __restrict__ planes, const Scalars* sc) {
  constexpr int RPB = PR_THREADS / T;  // rows per CTA
  constexpr int NS = UK / T;           // slots per thread
  __shared__ double Lt[UK][UK + 1];  // L_11 strictly below the diagonal; then the solved rows
  __shared__ double rcp[UK];
  if (*(volatile const int*)&sc->status != 0) return;  // a pivot of the diagonal factor failed
  for (int t = threadIdx.x; t < UK * UK; t += PR_THREADS) {  // the solve reads only Lt[i][j], j < i < kb
    const int i = t / UK, j = t % UK;
    Lt[i][j] = (j < i && i < kb) ? M[(k0 + i) * ldm + k0 + j] : 0.0;
  }
  for (int t = threadIdx.x; t < UK; t += PR_THREADS) rcp[t] = t < kb ? dinv[k0 + t] : 0.0;
  __syncthreads();
  const int row = threadIdx.x / T, part = threadIdx.x % T;
  const int64_t r0 = (int64_t)blockIdx.x * RPB;
  const bool live = r0 + row < rows;
  double* mrow = M + (live ? (k0 + kb + r0 + row) * ldm + k0 : 0);
  double x[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int c = part + T * k;
    x[k] = (live && c < kb) ? mrow[c] : 0.0;
  }
  // columns past kb hold zeros in B, L_11 and rcp: their slots stay zero
  const int src = (threadIdx.x & 31) - part;  // lane of this row's thread 0
#pragma unroll
  for (int c = 0; c < UK; ++c) {
    const int kc = c / T;
    const double own = x[kc];  // meaningful in the owner, part == c % T
    const double xc = __shfl_sync(0xffffffffu, own, src + c % T) * rcp[c];
    if (part == c % T) x[kc] = xc;
#pragma unroll
    for (int k = (c + 1) / T; k < NS; ++k) {
      if (T * k + T - 1 <= c) continue;  // no thread's slot k lies past c (compile-time)
      const int q = part + T * k;
      if (T * k > c || q > c) x[k] = fma(-xc, Lt[q][c], x[k]);
    }
  }
  __syncthreads();  // every thread is done with L_11
  double (*X)[UK + 1] = Lt;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int c = part + T * k;
    X[row][c] = c < kb ? x[k] : 0.0;
    if (live && c < kb) mrow[c] = x[k];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int rr = warp; rr < RPB; rr += PR_THREADS / 32) {
    const int64_t i = r0 + rr;
    if (i >= rows) break;
    const double v0 = X[rr][2 * lane], v1 = X[rr][2 * lane + 1];
    double mx = fmax(fabs(v0), fabs(v1));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int er = 0;
    if (mx > 0.0) frexp(mx, &er);
    if (lane == 0) e[i] = er;
    const double sc = ldexp(1.0, 55 - er);
    int d0[ND], d1[ND];
    balanced_digits(__double2ll_rn(v0 * sc), d0);
    balanced_digits(__double2ll_rn(v1 * sc), d1);
#pragma unroll
    for (int s = 0; s < ND; ++s) {
      const uint32_t pair = bf16_bits_small(d0[s]) | (bf16_bits_small(d1[s]) << 16);
      reinterpret_cast<uint32_t*>(planes + ((int64_t)s * mpad + i) * UK)[lane] = pair;
    }
  }
}

// FP64 warp instructions of one row-solve warp with T threads per row, and
// the warps of a panel of `rows` rows; the host takes the T with the
// smallest (warps per SM sub-partition, rounded up) x (instructions per warp).
constexpr int row_solve_instr(int T) {
  int n = UK;  // the x_c multiplies
  for (int c = 0; c < UK; ++c)
    for (int k = (c + 1) / T; k < UK / T; ++k)
      if (T * k + T - 1 > c) ++n;
  return n;
}

int pick_row_threads(int64_t rows, int sub_partitions) {
  const int Ts[4] = {4, 8, 16, 32};
  int best = 4;
  double best_cost = 1e300;
  for (int T : Ts) {
    const int64_t warps = (rows * T + 31) / 32;
    const int64_t per = (warps + sub_partitions - 1) / sub_partitions;
    const double cost = (double)per * row_solve_instr(T);
    if (cost < best_cost) {
      best_cost = cost;
      best = T;
    }
  }
  return best;
}

// Eight tensor-memory loads of 2 columns each (one per weight, w_stride
// columns apart) for this warp's 32 lanes, then one wait.
__device__ __forceinline__ void tmem_ld8x2(uint32_t taddr, uint32_t w_stride, uint32_t (&r)[NW][2]) {
#pragma unroll
  for (int w = 0; w < NW; ++w)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                 : "=r"(r[w][0]), "=r"(r[w][1])
                 : "r"(taddr + (uint32_t)w * w_stride));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Tile b of the update: (I, J) with J <= 4 I + 3 (row block I has 4 I + 4
// tiles, the first 2 I (I + 1) tiles precede it); false when the tile lies
// outside the trailing matrix.
__device__ __forceinline__ bool update_tile(int64_t b, int64_t rows, int64_t& p0, int64_t& q0) {
  int64_t I = (int64_t)((sqrtf(2.0f * (float)b + 1.0f) - 1.0f) * 0.5f);  // FP32 estimate, corrected below
  while (2 * I * (I + 1) > b) --I;
  while (2 * (I + 1) * (I + 2) <= b) ++I;
  p0 = I * UBM;
  q0 = (b - 2 * I * (I + 1)) * UBN;
  return q0 < rows && q0 <= p0 + UBM - 1;
}

// C_pq -= (P P')_pq for the lower tiles of the trailing matrix (rows and
// columns base + [0, rows)).  Persistent: CTA x takes a contiguous range of
// tiles, so consecutive tiles share their row block and its P planes (copied
// once per row block).  Two tiles are in flight: the Q planes and the
// accumulators are double-buffered, so the MMAs of tile i + 1 run while the
// epilogue reads and writes back tile i.
__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_dig_update(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmQ, int64_t ldm,
                 double* __restrict__ M, int64_t base, int64_t rows, int64_t ntiles, const int* __restrict__ e,
                 double* __restrict__ dinv, int kbn, Scalars* sc) {
  extern __shared__ uint8_t smem_raw[];
  if (*(volatile const int*)&sc->status != 0) return;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  // barriers: P full | P free | Q full[2] | Q free[2] | MMA done[2] | TMEM free[2] | drain
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + LOAD_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 11);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* diag_go = reinterpret_cast<volatile int*>(tmem_slot + 2);
  double* stage_all = reinterpret_cast<double*>(smem + LOAD_BYTES + 256);
  const uint32_t pfull = smem_u32(bars), pfree = smem_u32(bars + 1), drain = smem_u32(bars + 10);
  auto qfull = [&](int b) { return smem_u32(bars + 2 + b); };
  auto qfree = [&](int b) { return smem_u32(bars + 4 + b); };
  auto mma_done = [&](int b) { return smem_u32(bars + 6 + b); };
  auto tfree = [&](int b) { return smem_u32(bars + 8 + b); };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(pfull, 1);
    mbar_init(pfree, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(qfull(b), 1);
      mbar_init(qfree(b), 1);
      mbar_init(mma_done(b), 1);
      mbar_init(tfree(b), EPI_WARPS);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  int64_t p0, q0;
  // this CTA's tiles [tb, te).  With the next panel's diagonal block folded
  // in (kbn > 0), CTA 0 takes tiles 0 and 1 alone (rows 0..127, columns
  // 0..63: they hold that block) and factors the block once they are
  // written; the other CTAs share the rest in equal contiguous ranges.
  const bool fold = kbn > 0;
  int64_t tb, te;
  if (fold && gridDim.x > 1) {
    const int64_t head = ntiles < 2 ? ntiles : 2, rest = ntiles - head, g = gridDim.x - 1;
    tb = blockIdx.x == 0 ? 0 : head + rest * (blockIdx.x - 1) / g;
    te = blockIdx.x == 0 ? head : head + rest * blockIdx.x / g;
  } else {
    tb = ntiles * blockIdx.x / gridDim.x;
    te = ntiles * (blockIdx.x + 1) / gridDim.x;
  }

  if (warp == 0) {
    if (lane == 0) {
      int i = 0, pl = 0;  // tiles and P copies issued
      int64_t cur = -1;   // row block of the P planes in shared memory
      for (int64_t b = tb; b < te; ++b) {
        if (!update_tile(b, rows, p0, q0)) continue;
        if (p0 != cur) {  // a new row block: its P planes, once the last one's MMAs are done
          if (pl > 0 && !mbar_wait(pfree, (uint32_t)(pl - 1) & 1u, abort_flag)) {
            *abort_flag = 1;
            break;
          }
          mbar_expect_tx(pfull, P_BYTES);
          tma_load_3d(sbase, &tmP, 0, (int)p0, 0, pfull);
          cur = p0;
          ++pl;
        }
        const int bf = i & 1;
        if (i >= 2 && !mbar_wait(qfree(bf), (uint32_t)((i >> 1) - 1) & 1u, abort_flag)) {
          *abort_flag = 1;
          break;
        }
        mbar_expect_tx(qfull(bf), Q_BYTES);
        tma_load_3d(sbase + P_BYTES + (uint32_t)bf * Q_BYTES, &tmQ, 0, (int)q0, 0, qfull(bf));
        ++i;
      }
      // every issued copy has landed before the CTA can leave
      if (pl > 0) mbar_wait(pfull, (uint32_t)(pl - 1) & 1u, nullptr);
      for (int k = i > 2 ? i - 2 : 0; k < i; ++k) mbar_wait(qfull(k & 1), (uint32_t)(k >> 1) & 1u, nullptr);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      int i = 0, pl = 0;
      int64_t cur = -1;
      for (int64_t b = tb; b < te && !*abort_flag; ++b) {
        if (!update_tile(b, rows, p0, q0)) continue;
        const int bf = i & 1;
        if (p0 != cur) {
          if (cur >= 0) umma_commit(pfree);  // the last row block's MMAs: its P planes may be overwritten
          if (!mbar_wait(pfull, (uint32_t)pl & 1u, abort_flag)) {
            *abort_flag = 1;
            break;
          }
          cur = p0;
          ++pl;
        }
        if (!mbar_wait(qfull(bf), (uint32_t)(i >> 1) & 1u, abort_flag) ||
            (i >= 2 && !mbar_wait(tfree(bf), (uint32_t)((i >> 1) - 1) & 1u, abort_flag))) {
          *abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t qb = sbase + P_BYTES + (uint32_t)bf * Q_BYTES;
        const uint32_t dbuf = tmem + (uint32_t)bf * BUF_COLS;
#pragma unroll
        for (int g = 0; g < NGROUP; ++g) {
          const MmaGroup G = mma_group(g);
          const uint64_t ad = sdesc_sw128(sbase + G.s * P_PLANE);
          const uint64_t bd = sdesc_sw128(qb + G.t0 * Q_PLANE);
          const uint32_t d = dbuf + (uint32_t)((G.s + G.t0) * UBN);
          const uint32_t idesc = idesc_bf16(UBM, UBN * G.nt);
#pragma unroll
          for (int k = 0; k < 4; ++k)  // 32 bytes (16 BF16) along K per MMA
            umma_f16(d, ad + 2 * k, bd + 2 * k, idesc, G.first && k == 0 ? 0u : 1u);
        }
        umma_commit(qfree(bf));     // the Q planes may be overwritten once these MMAs are done
        umma_commit(mma_done(bf));  // and the accumulators read
        ++i;
      }
      umma_commit(drain);  // every MMA issued above has completed before the CTA leaves
      mbar_wait(drain, 0, nullptr);
    }
    __syncwarp();
  } else {
    constexpr int EC = UBN / (EPI_WARPS / 4);  // columns per epilogue warp: 8
    static_assert(EC == 8, "one staging round of 8 columns per tile");
    const int quarter = warp & 3, cg = (warp - 2) >> 2;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cg * EC);
    double* stg = stage_all + (warp - 2) * 32 * STG_PITCH;
    int i = 0;
    for (int64_t b = tb; b < te; ++b) {
      if (!update_tile(b, rows, p0, q0)) continue;
      const int bf = i & 1;
      // this warp's block: rows p0 + 32 quarter + [0, 32) (row p = lane in
      // tensor memory), columns qb + [0, 8), those with q <= p inside the
      // trailing matrix
      const int64_t rw = p0 + quarter * 32;
      const int64_t p = rw + lane;
      const int64_t qb = q0 + cg * EC;
      const bool prow = p < rows;
      const int ep = prow ? e[p] : 0;
      const int eq_lane = lane < EC && qb + lane < rows ? e[qb + lane] : 0;  // e_q of column qb + lane, by shuffles
      // C is read and written in a coalesced layout: lane l takes column
      // qb + (l & 7) of rows rw + (l >> 3) + 4 k, k < 8 (four 64-byte row
      // segments per access).  The loads are issued before the wait, so they
      // are in flight while the tile's MMAs run (C does not depend on them).
      const int cl = lane & 7, rl = lane >> 3;
      double cc[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int64_t r = rw + rl + 4 * k, q = qb + cl;
        cc[k] = (r < rows && q <= r) ? M[(base + r) * ldm + base + q] : 0.0;
      }
      int ok = 1;
      if (lane == 0) ok = mbar_wait(mma_done(bf), (uint32_t)(i >> 1) & 1u, abort_flag) && !*abort_flag;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) *abort_flag = 1;
        break;
      }
      fence_after();
      // GB300 runs FP64 at 1/64 of the FP32 rate, so the weights are
      // combined on the integer pipes into one integer per entry,
      //   Z = sum_{w<=5} I_w 2^(42-8w) + round((I_6 2^8 + I_7) 2^-14)
      //     = t_01 2^34 + t_23 2^18 + t_45 2^2 + round(t_67 2^-14),
      //   t_ab = I_a 2^8 + I_b, exact in int32 (|I_w| <= 7 2^20)
      // (|I_0| <= 2^20: |Z| < 2^63; the rounding is 2^-43 of
      // sum_w 2^-8w I_w, below the digits' own truncation).  All of the
      // tile's accumulators are read first, so the MMAs of tile i + 2 can
      // start; Z 2^(e_p + e_q - 56) is then built as a double on the integer
      // pipes and subtracted from C (the one FP64 operation of an entry).
      long long Z[EC];
#pragma unroll
      for (int g = 0; g < EC / 2; ++g) {  // 2 columns at a time
        uint32_t r[NW][2];
        tmem_ld8x2(lane_addr + (uint32_t)bf * BUF_COLS + (uint32_t)(g * 2), UBN, r);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          // weights 0..3 collect at most 4 pairs: |I_w| <= 2^22, so the FP32
          // sum I_w + 1.5 2^23 is exact and its bits minus those of 1.5 2^23
          // are I_w (an add on the FMA pipe); weights 4..7 through the
          // conversion pipe
          int iw[NW];
#pragma unroll
          for (int w = 0; w < NW; ++w)
            iw[w] = w < 4 ? __float_as_int(__uint_as_float(r[w][j]) + 12582912.0f) - 0x4B400000
                          : __float2int_rn(__uint_as_float(r[w][j]));
          const int t01 = iw[0] * 256 + iw[1], t23 = iw[2] * 256 + iw[3], t45 = iw[4] * 256 + iw[5];
          const int t67 = iw[6] * 256 + iw[7];
          Z[g * 2 + j] = (long long)t01 * (1ll << 34) + (long long)t23 * (1ll << 18) + (long long)t45 * 4 +
                         ((t67 + 8192) >> 14);
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tfree(bf));  // the accumulators may be overwritten
      // the updates of row p (this lane) go through the warp's staging area
#pragma unroll
      for (int c = 0; c < EC; ++c) {
        const int eqc = __shfl_sync(0xffffffffu, eq_lane, c);
        stg[lane * STG_PITCH + c] = (prow && qb + c <= p) ? scaled_int_to_double(Z[c], ep + eqc - 56) : 0.0;
      }
      __syncwarp();
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int64_t r = rw + rl + 4 * k, q = qb + cl;
        if (r < rows && q <= r) M[(base + r) * ldm + base + q] = cc[k] - stg[(rl + 4 * k) * STG_PITCH + cl];
      }
      __syncwarp();
      ++i;
    }
    if (fold && blockIdx.x == 0) {
      // tiles 0 and 1 are written (the barrier orders every epilogue
      // thread's stores before the reads below) and their MMAs are done, so
      // the plane buffer is free: the epilogue warps factor the next panel's
      // diagonal block there, if no wait of this CTA gave up (one thread
      // decides, all follow)
      asm volatile("bar.sync 1, %0;" ::"r"(EPI_WARPS * 32) : "memory");
      if (threadIdx.x == 64) *diag_go = !*abort_flag;
      asm volatile("bar.sync 1, %0;" ::"r"(EPI_WARPS * 32) : "memory");
      if (*diag_go)
        diag_factor<EPI_WARPS * 32>(ldm, M, dinv, base, kbn, sc, *reinterpret_cast<DiagSmem*>(smem),
                                    (int)threadIdx.x - 64,
                                    [] { asm volatile("bar.sync 1, %0;" ::"r"(EPI_WARPS * 32) : "memory"); });
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
static_assert(sizeof(DiagSmem) <= LOAD_BYTES, "the folded diagonal factor fits the plane buffer");

struct CholDigHost {
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  CUtensorMap mapP, mapQ;
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

// 3-D map over the 7 digit planes: dims {64, mpad, 7}, box {64, rows, 7},
// 128-byte swizzle; the box lands as 7 x rows x 128 B.
cudaError_t encode_planes(CholDigHost* hs, CUtensorMap* map, const void* base, int64_t mpad, int rows) {
  cuuint64_t dims[3] = {(cuuint64_t)UK, (cuuint64_t)mpad, (cuuint64_t)ND};
  cuuint64_t strides[2] = {(cuuint64_t)(UK * 2), (cuuint64_t)(mpad * UK * 2)};
  cuuint32_t box[3] = {(cuuint32_t)UK, (cuuint32_t)rows, (cuuint32_t)ND};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = hs->encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t chol_dig_create(CholDigWorkspace* w, int64_t m) {
  w->m = m;
  w->mpad = (m + UBM - 1) / UBM * UBM;
  int dev = 0, sms = 0;
  cudaError_t ea = cudaGetDevice(&dev);
  if (ea == cudaSuccess) ea = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (ea != cudaSuccess) return ea;
  w->sub_partitions = 4 * sms;
  CholDigHost* hs = new (std::nothrow) CholDigHost();
  if (!hs) return cudaErrorMemoryAllocation;
  w->host = hs;
  cudaError_t e = get_encoder(&hs->encode);
  const size_t plane_bytes = sizeof(__nv_bfloat16) * (size_t)ND * w->mpad * UK;
  if (e == cudaSuccess) e = cudaMalloc(&w->planes, plane_bytes);
  if (e == cudaSuccess) e = cudaMemset(w->planes, 0, plane_bytes);  // rows never written read as 0
  if (e == cudaSuccess) e = cudaMalloc(&w->e, sizeof(int) * (size_t)w->mpad);
  if (e == cudaSuccess) e = cudaMemset(w->e, 0, sizeof(int) * (size_t)w->mpad);
  if (e == cudaSuccess) e = encode_planes(hs, &hs->mapP, w->planes, w->mpad, UBM);
  if (e == cudaSuccess) e = encode_planes(hs, &hs->mapQ, w->planes, w->mpad, UBN);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dig_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  return e;
}

void chol_dig_destroy(CholDigWorkspace* w) {
  if (w->planes) cudaFree(w->planes);
  if (w->e) cudaFree(w->e);
  delete static_cast<CholDigHost*>(w->host);
  *w = CholDigWorkspace{};
}

cudaError_t cholesky_dig(cudaStream_t st, CholDigWorkspace* w, int64_t ldm, double* M, double* dinv, Scalars* sc,
                         int* launches) {
  *launches = 0;
  const int64_t m = w->m;
  CholDigHost* hs = static_cast<CholDigHost*>(w->host);
  cudaError_t e = cudaSuccess;
  for (int64_t k0 = 0; k0 < m && e == cudaSuccess; k0 += UK) {
    const int kb = (int)std::min<int64_t>(UK, m - k0);
    const int64_t rows = m - k0 - kb;  // the trailing matrix
    if (k0 == 0) {  // later diagonal blocks are factored inside the previous panel's update
      k_dig_diag<<<1, DG_THREADS, 0, st>>>(ldm, M, dinv, k0, kb, sc);
      ++*launches;
      e = cudaGetLastError();
    }
    if (e != cudaSuccess || rows == 0) continue;
    __nv_bfloat16* planes = static_cast<__nv_bfloat16*>(w->planes);
    switch (pick_row_threads(rows, w->sub_partitions)) {
      case 4:
        k_dig_panel_rows<4><<<(unsigned)((rows + 31) / 32), PR_THREADS, 0, st>>>(ldm, M, dinv, k0, kb, rows, w->mpad,
                                                                                 w->e, planes, sc);
        break;
      case 8:
        k_dig_panel_rows<8><<<(unsigned)((rows + 15) / 16), PR_THREADS, 0, st>>>(ldm, M, dinv, k0, kb, rows, w->mpad,
                                                                                 w->e, planes, sc);
        break;
      case 16:
        k_dig_panel_rows<16><<<(unsigned)((rows + 7) / 8), PR_THREADS, 0, st>>>(ldm, M, dinv, k0, kb, rows, w->mpad,
                                                                                w->e, planes, sc);
        break;
      default:
        k_dig_panel_rows<32><<<(unsigned)((rows + 3) / 4), PR_THREADS, 0, st>>>(ldm, M, dinv, k0, kb, rows, w->mpad,
                                                                                w->e, planes, sc);
    }
    const int64_t nI = (rows + UBM - 1) / UBM, ntiles = 2 * nI * (nI + 1);
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, w->sub_partitions / 4);
    const int kbn = (int)std::min<int64_t>(UK, rows);  // the next panel's width: its diagonal block is folded in
    k_dig_update<<<grid, NUM_THREADS, SMEM_BYTES, st>>>(hs->mapP, hs->mapQ, ldm, M, k0 + kb, rows, ntiles, w->e,
                                                        dinv, kbn, sc);
    *launches += 2;
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace pdas
