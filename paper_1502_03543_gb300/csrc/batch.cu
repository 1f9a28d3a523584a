// batch.cu -- many small LPs by the PDAS algorithm (Section III, Newton
// direction of Section V), one CTA per LP, in one persistent launch per size
// bucket (pdas_batch.h).
//
// A CTA runs its LP's whole iteration loop:
//   D = x/s;  r = A x;  M = (A D^1/2)(A D^1/2)' (FP32, lower triangle packed
//   in shared memory);  M = L L' (FP32, in shared memory; once a pivot is
//   not positive, the LP continues with M formed in double-float and factored
//   in FP64 in a global scratch slot of its CTA, as the large path does near
//   the optimum);  dy = L'^-1 L^-1 r;  preconditioned conjugate
//   gradients on the exact M (matrix-free, double-float products on the FP32
//   pipes, FP64 vectors) until ||r - M dy|| meets the tolerance;
//   w = A' dy, dx = D w - x, ds = -w;  psi, theta = alpha/psi (1 if psi <= 1);
//   the step; the relative gap.
// All reductions are block-level with a fixed order, so results do not
// depend on which CTA or in which order the LPs run.
//
// GB300 issues FP64 at 1/64 of its FP32 rate; the passes A v (r = A x and
// the outer product of M v) run in double-float (df_util.cuh), about FP64
// accurate, while the passes A' v stay FP64 because D multiplies their result
// (see blk_gemv_t).  M and its factor are FP32 as in the FP32 mixed form of
// the large path.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "df_util.cuh"
#include "pdas_batch.h"
#include "reduce_util.cuh"

namespace pdas {

namespace {

struct BatchLP {
  int m, n;
  int64_t a_off, m_off, n_off;
};

struct BatchArgs {
  const BatchLP* lps;
  const int* order;  // LP indices of the bucket, largest first
  int count;         // LPs in the bucket
  int m_cap, n_cap;  // shared-memory capacity of the launch
  const float* A;
  const double* b;
  const double* c;
  double* x;
  double* y;
  double* s;
  double alpha, tol, refine_tol;
  int max_iter, refine_max;
  int* status;
  int* iters;
  double* gap;
  int* shifted;    // iterations run with the FP64 factor (after the FP32 factor failed)
  int* unrefined;  // iterations whose refinement stopped without meeting refine_tol
  float* time_us;  // device time of each LP's solve
  unsigned* ticket;
  double* scratch;  // FP64 tier: per CTA slot, packed lower M / L then 1 / L_pp
  int64_t slot;     // doubles per slot: m_cap (m_cap + 1) / 2 + m_cap
};

// Shared-memory layout for capacities (mc, nc): 16-byte aligned sections.
struct BatchSmem {
  size_t L, dinv, zf, vm, pm2, D, w, un2, kidx, stage, dc, scal, total;
};
__host__ __device__ inline size_t al16(size_t v) { return (v + 15) & ~size_t(15); }
__host__ __device__ inline BatchSmem batch_smem(int mc, int nc) {
  BatchSmem o;
  size_t p = 0;
  o.L = p;     p = al16(p + sizeof(float) * (size_t)mc * (mc + 1) / 2);
  o.dinv = p;  p = al16(p + sizeof(float) * mc);
  o.zf = p;    p = al16(p + sizeof(float) * mc);
  o.vm = p;    p = al16(p + sizeof(double) * 6 * mc);
  o.pm2 = p;   p = al16(p + sizeof(float2) * mc);
  o.D = p;     p = al16(p + sizeof(double) * nc);
  o.w = p;     p = al16(p + sizeof(double) * nc);
  o.un2 = p;   p = al16(p + sizeof(float2) * nc);
  o.kidx = p;  p = al16(p + sizeof(int) * nc);
  o.stage = p; p = al16(p + sizeof(float) * mc * 34);  // (also an FP64 panel of 16 columns, pitch 17)
  o.dc = p;    p = al16(p + sizeof(float) * 64);
  o.scal = p;  p = al16(p + sizeof(double) * 32);
  o.total = p;
  return o;
}

// packed lower-triangle index of (r, q), q <= r
__device__ __forceinline__ int pk(int r, int q) { return r * (r + 1) / 2 + q; }

__device__ __forceinline__ float inv_sqrt32(float d) {
  const float r = rsqrtf(d);
  return r * fmaf(-0.5f * d * r, r, 1.5f);
}

// Per-CTA view of the shared memory and of the current LP.
struct Ctx {
  float* L;      // packed lower triangle of M, then of its factor
  float* dinv;   // 1 / L_pp
  float* zf;     // FP32 vector of the triangular solves
  double* r;     // A x
  double* dy;    // direction
  double* rho;   // refinement residual
  double* z;     // preconditioned residual
  double* p;     // search direction
  double* q;     // M p
  double* D;     // x / s
  double* w;     // A' (an m-vector)
  float2* un2;   // an n-vector as FP32 pairs
  float2* pm2;   // an m-vector as FP32 pairs
  int* kidx;     // FP64 tier: the columns kept for the normal matrix
  float* stage;  // [m_cap][33]: 32 columns of A D^1/2
  float* dc;     // 32 entries of D^1/2, or of D as FP32 pairs (64 floats)
  double* scal;  // reduction scratch
  const float* A;
  int m, n;
};

template <int T>
__device__ __forceinline__ double bsum(double v, double* scal) {
  const double t = block_reduce<0>(v, scal);
  __syncthreads();
  if (threadIdx.x == 0) scal[0] = t;
  __syncthreads();
  const double r = scal[0];
  __syncthreads();
  return r;
}
template <int T>
__device__ __forceinline__ double bmax(double v, double* scal) {
  const double t = block_reduce<1>(v, scal);
  __syncthreads();
  if (threadIdx.x == 0) scal[0] = t;
  __syncthreads();
  const double r = scal[0];
  __syncthreads();
  return r;
}

// out_p = [base_p -] A_p. v for the FP32-pair vector v2 (n); one warp per row.
template <int T>
__device__ void blk_gemv(const Ctx& c, const float2* v2, const double* base, double* out) {
  constexpr int NW = T / 32;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int p = wp; p < c.m; p += NW) {
    const float* row = c.A + (int64_t)p * c.n;
    double acc = 0.0;
    float hi = 0.f, lo = 0.f;
    for (int j0 = lane; j0 < c.n; j0 += 32 * 8) {  // 8 loads in flight per lane
      float av[8];
      float2 vv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + 32 * u;
        av[u] = j < c.n ? __ldg(row + j) : 0.f;
        vv[u] = j < c.n ? v2[j] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) df_madd(hi, lo, av[u], vv[u].x, vv[u].y);
      df_flush(acc, hi, lo);
    }
    acc = warp_sum(acc);
    if (lane == 0) out[p] = base ? base[p] - acc : acc;
  }
}

// out_j = sum_p A_pj u_p in FP64 (exact widening of A on the integer pipes,
// FP64 multiply-adds); one thread per column.  Every use of A' (.) here is
// multiplied by D afterwards (dx = D w - x, u = D A' v), which spans many
// orders of magnitude near the optimum, so this pass keeps FP64 accuracy.
template <int T>
__device__ void blk_gemv_t(const Ctx& c, const double* u, double* out) {
  for (int j = threadIdx.x; j < c.n; j += T) {
    const float* col = c.A + j;
    double acc = 0.0;
    for (int p0 = 0; p0 < c.m; p0 += 8) {  // 8 loads in flight per thread
      float av[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) av[k] = p0 + k < c.m ? __ldg(col + (int64_t)(p0 + k) * c.n) : 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (p0 + k < c.m) acc = fma(widen_bits(__float_as_uint(av[k])), u[p0 + k], acc);
    }
    out[j] = acc;
  }
}

// M = (A D^1/2)(A D^1/2)' into c.L (packed lower), FP32: 32-column chunks of
// A D^1/2 staged in shared memory; warps take 32 x 32 lower tiles, a lane
// holding rows lr + 8 i (i < 4) and columns lc + 4 j (j < 8) of its tile.
// m_cap is a multiple of 32, so every staged row index is in range; rows past
// m are staged as zero.
template <int T>
__device__ void blk_syrk(const Ctx& c, int m_cap) {
  constexpr int NW = T / 32;
  const int m = c.m, n = c.n;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, lr = lane >> 2, lc = lane & 3;
  const int mt = (m + 31) >> 5, ntile = mt * (mt + 1) / 2;
  for (int e = threadIdx.x; e < m * (m + 1) / 2; e += T) c.L[e] = 0.f;
  for (int k0 = 0; k0 < n; k0 += 32) {
    if (threadIdx.x < 32) c.dc[threadIdx.x] = k0 + threadIdx.x < n ? (float)sqrt(c.D[k0 + threadIdx.x]) : 0.f;
    __syncthreads();
    for (int e = threadIdx.x; e < m_cap * 32; e += T) {
      const int r = e >> 5, kk = e & 31;
      c.stage[r * 33 + kk] = (r < m && k0 + kk < n) ? __ldg(c.A + (int64_t)r * n + k0 + kk) * c.dc[kk] : 0.f;
    }
    __syncthreads();
    for (int t = wp; t < ntile; t += NW) {
      int tp = 0;
      while ((tp + 1) * (tp + 2) / 2 <= t) ++tp;
      const int tq = t - tp * (tp + 1) / 2;
      float acc[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 4
      for (int kk = 0; kk < 32; ++kk) {
        float a[4], bb[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = c.stage[(tp * 32 + lr + 8 * i) * 33 + kk];
#pragma unroll
        for (int j = 0; j < 8; ++j) bb[j] = c.stage[(tq * 32 + lc + 4 * j) * 33 + kk];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int pr = tp * 32 + lr + 8 * i;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int qc = tq * 32 + lc + 4 * j;
          if (pr < m && qc <= pr) c.L[pk(pr, qc)] += acc[i][j];
        }
      }
    }
    __syncthreads();
  }
}

// In-place Cholesky of the packed lower triangle (FP32), right-looking by
// columns, two block barriers per column; the scaled column is read from a
// contiguous copy (zf) in the trailing update.  Returns false on a pivot that is
// not positive and finite (the same in every thread).
template <int T>
__device__ bool blk_chol(const Ctx& c) {
  constexpr int NW = T / 32;
  const int m = c.m, lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int k = 0; k < m; ++k) {
    __syncthreads();
    const float d = c.L[pk(k, k)];
    if (!(d > 0.f) || !isfinite(d)) return false;
    const float rs = inv_sqrt32(d);
    for (int r = k + 1 + threadIdx.x; r < m; r += T) {  // the scaled column, also kept in zf
      const float v = c.L[pk(r, k)] * rs;
      c.L[pk(r, k)] = v;
      c.zf[r] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      c.L[pk(k, k)] = d * rs;
      c.dinv[k] = rs;
    }
    for (int r = k + 1 + wp; r < m; r += NW) {
      const float lrk = c.zf[r];
      float* row = c.L + pk(r, 0);
      for (int q = k + 1 + lane; q <= r; q += 32) row[q] = fmaf(-lrk, c.zf[q], row[q]);
    }
  }
  __syncthreads();
  return true;
}

// out = (L L')^{-1} v (FP64 in and out, FP32 solves by warp 0; the rows of
// the vector are spread over the lanes, the pivot entry is read by all).
template <int T>
__device__ void blk_precond(const Ctx& c, const double* v, double* out) {
  const int m = c.m, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < m; i += T) c.zf[i] = (float)v[i];
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int r = 0; r < m; ++r) {  // L z = v, row by row (contiguous packed rows)
      const float* row = c.L + pk(r, 0);
      float t = 0.f;
      for (int k = lane; k < r; k += 32) t = fmaf(row[k], c.zf[k], t);
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) c.zf[r] = (c.zf[r] - t) * c.dinv[r];
      __syncwarp();
    }
    for (int k = m - 1; k >= 0; --k) {  // L' y = z
      const float yk = c.zf[k] * c.dinv[k];
      for (int r = lane; r < k; r += 32) c.zf[r] = fmaf(-c.L[pk(k, r)], yk, c.zf[r]);
      __syncwarp();
      if (lane == 0) c.zf[k] = yk;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += T) out[i] = (double)c.zf[i];
  __syncthreads();
}

// ---- the FP64 tier: M and L (FP64) in the CTA's global scratch slot ----

// M_K = A_K D_K A_K' (FP64, packed lower) over the nk columns listed in
// kidx, in double-float on the FP32 pipes: 32-column chunks of A_K staged as
// in blk_syrk (unscaled), D_k as an FP32 pair,
// (A_qk D_k) split exactly by FMA, the products accumulated as FP32 pairs
// over the chunk and flushed into FP64 once per chunk.
template <int T>
__device__ void blk_syrk_df(const Ctx& c, int m_cap, double* M, int nk) {
  constexpr int NW = T / 32;
  const int m = c.m, n = nk;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, lr = lane >> 2, lc = lane & 3;
  const int mt = (m + 31) >> 5, ntile = mt * (mt + 1) / 2;
  for (int e = threadIdx.x; e < m * (m + 1) / 2; e += T) M[e] = 0.0;
  for (int k0 = 0; k0 < n; k0 += 32) {
    if (threadIdx.x < 32) {
      const float2 d = k0 + threadIdx.x < n ? df_split(c.D[c.kidx[k0 + threadIdx.x]]) : make_float2(0.f, 0.f);
      c.dc[threadIdx.x] = d.x;
      c.dc[32 + threadIdx.x] = d.y;
    }
    for (int e = threadIdx.x; e < m_cap * 32; e += T) {
      const int r = e >> 5, kk = e & 31;
      c.stage[r * 33 + kk] = (r < m && k0 + kk < n) ? __ldg(c.A + (int64_t)r * c.n + c.kidx[k0 + kk]) : 0.f;
    }
    __syncthreads();
    for (int t = wp; t < ntile; t += NW) {
      int tp = 0;
      while ((tp + 1) * (tp + 2) / 2 <= t) ++tp;
      const int tq = t - tp * (tp + 1) / 2;
      float hi[4][8], lo[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) hi[i][j] = lo[i][j] = 0.f;
#pragma unroll 1
      for (int kk = 0; kk < 32; ++kk) {
        const float dh = c.dc[kk], dl = c.dc[32 + kk];
        float a[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = c.stage[(tp * 32 + lr + 8 * i) * 33 + kk];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float aq = c.stage[(tq * 32 + lc + 4 * j) * 33 + kk];
          const float bh = aq * dh;
          const float bl = fmaf(aq, dl, fmaf(aq, dh, -bh));
#pragma unroll
          for (int i = 0; i < 4; ++i) df_madd(hi[i][j], lo[i][j], a[i], bh, bl);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int pr = tp * 32 + lr + 8 * i;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int qc = tq * 32 + lc + 4 * j;
          if (pr < m && qc <= pr) {
            double acc = M[pk(pr, qc)];
            df_flush(acc, hi[i][j], lo[i][j]);
            M[pk(pr, qc)] = acc;
          }
        }
      }
    }
    __syncthreads();
  }
}

// In-place FP64 Cholesky of the packed lower triangle in global memory, in
// panels of 16 columns: the panel (rows k0.. m-1) is factored in shared
// memory (the stage area, pitch 17 doubles), written back, and the trailing
// lower triangle is updated once per panel (16 multiply-adds per entry, one
// read-modify-write of global memory).  dinv receives 1 / L_kk.  Returns
// false on a pivot that is not positive and finite.
// The pivot's square root and reciprocal are formed once, by thread 0 (which
// updates the next diagonal entry first), and passed on in shared memory:
// FP64 runs at a small fraction of the FP32 rate, and the same two
// operations in every thread would cost more than the column's update.
__device__ __forceinline__ void post_pivot(double d, double* slot) {
  const bool ok = d > 0.0 && isfinite(d);
  const double lkk = ok ? sqrt(d) : -1.0;
  slot[0] = lkk;
  slot[1] = ok ? 1.0 / lkk : 0.0;
}

template <int T>
__device__ bool blk_chol64(const Ctx& c, double* L, double* dinv) {
  constexpr int NW = T / 32, PW = 16, PP = 17;
  __shared__ double piv[2][2];  // (L_kk, 1 / L_kk) of the next two columns; L_kk < 0: not positive definite
  const int m = c.m, lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  double* P = reinterpret_cast<double*>(c.stage);
  for (int k0 = 0; k0 < m; k0 += PW) {
    const int kb = m - k0 < PW ? m - k0 : PW, R = m - k0;
    __syncthreads();
    for (int e = threadIdx.x; e < R * PW; e += T) {
      const int r = e / PW, cc = e % PW;
      P[r * PP + cc] = (cc < kb && cc <= r) ? L[pk(k0 + r, k0 + cc)] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) post_pivot(P[0], piv[0]);
    __syncthreads();
    for (int cc = 0; cc < kb; ++cc) {
      const double lkk = piv[cc & 1][0], rs = piv[cc & 1][1];
      if (lkk < 0.0) return false;
      for (int r = cc + 1 + threadIdx.x; r < R; r += T) P[r * PP + cc] *= rs;
      __syncthreads();
      if (threadIdx.x == 0) {
        P[cc * PP + cc] = lkk;
        dinv[k0 + cc] = rs;
      }
      const int nc = kb - cc - 1;  // later panel columns
      for (int e = threadIdx.x; e < (R - cc - 1) * nc; e += T) {
        const int r = cc + 1 + e / nc, q = cc + 1 + e % nc;
        if (q <= r) {
          P[r * PP + q] = fma(-P[r * PP + cc], P[q * PP + cc], P[r * PP + q]);
          if (e == 0) post_pivot(P[r * PP + q], piv[(cc + 1) & 1]);  // thread 0: entry (cc + 1, cc + 1)
        }
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < R * kb; e += T) {
      const int r = e / kb, cc = e % kb;
      if (cc <= r) L[pk(k0 + r, k0 + cc)] = P[r * PP + cc];
    }
    for (int r = kb + wp; r < R; r += NW) {  // trailing: L_rq -= sum_c P_rc P_qc
      double pr[PW];
#pragma unroll
      for (int cc = 0; cc < PW; ++cc) pr[cc] = P[r * PP + cc];
      double* row = L + pk(k0 + r, k0);
      for (int q = kb + lane; q <= r; q += 32) {
        double v = row[q];
#pragma unroll
        for (int cc = 0; cc < PW; ++cc) v = fma(-pr[cc], P[q * PP + cc], v);
        row[q] = v;
      }
    }
  }
  __syncthreads();
  return true;
}

// out = (L L')^{-1} v with the FP64 factor: forward substitution row by row
// (a warp dot product over the contiguous packed row), back substitution by
// rows of L (a warp sweep); out must not alias v.
template <int T>
__device__ void blk_precond64(const Ctx& c, const double* L, const double* dinv, const double* v, double* out) {
  const int m = c.m, lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    for (int r = 0; r < m; ++r) {  // L z = v
      const double* row = L + pk(r, 0);
      double t = 0.0;
      for (int k = lane; k < r; k += 32) t = fma(row[k], out[k], t);
      t = warp_sum(t);
      if (lane == 0) out[r] = (v[r] - t) * dinv[r];
      __syncwarp();
    }
    for (int k = m - 1; k >= 0; --k) {  // L' y = z
      const double yk = out[k] * dinv[k];
      const double* row = L + pk(k, 0);
      for (int r = lane; r < k; r += 32) out[r] = fma(-row[r], yk, out[r]);
      __syncwarp();
      if (lane == 0) out[k] = yk;
      __syncwarp();
    }
  }
  __syncthreads();
}

// out_j = sum_p A_pj u_p in double-float for the FP32-pair vector u2 (m);
// one thread per column.  Used for the conjugate-gradient operator while the
// factor is FP32, where D spans fewer orders of magnitude.
template <int T>
__device__ void blk_gemv_t_df(const Ctx& c, const float2* u2, double* out) {
  for (int j = threadIdx.x; j < c.n; j += T) {
    const float* col = c.A + j;
    double acc = 0.0;
    float hi = 0.f, lo = 0.f;
    for (int p0 = 0; p0 < c.m; p0 += 8) {  // 8 loads in flight per thread
      float av[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) av[u] = p0 + u < c.m ? __ldg(col + (int64_t)(p0 + u) * c.n) : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float2 q = p0 + u < c.m ? u2[p0 + u] : make_float2(0.f, 0.f);
        df_madd(hi, lo, av[u], q.x, q.y);
      }
      if ((p0 & 15) == 8) df_flush(acc, hi, lo);
    }
    df_flush(acc, hi, lo);
    out[j] = acc;
  }
}

// out = M v = A (D (A' v)), FP64 result; the outer pass in double-float, the
// inner one in FP64 (or double-float when df_inner).  Leaves w = A' v.
// (base != null: out = base - M v.)
template <int T>
__device__ void blk_apply_m(const Ctx& c, const double* v, const double* base, double* out, bool df_inner = false) {
  if (df_inner) {
    for (int i = threadIdx.x; i < c.m; i += T) c.pm2[i] = df_split(v[i]);
    __syncthreads();
    blk_gemv_t_df<T>(c, c.pm2, c.w);
  } else {
    blk_gemv_t<T>(c, v, c.w);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < c.n; j += T) c.un2[j] = df_split(c.D[j] * c.w[j]);
  __syncthreads();
  blk_gemv<T>(c, c.un2, base, out);
  __syncthreads();
}

// M at the current D and its factor.  Until an FP32 factor fails (tier2
// false) M is formed and factored in FP32 in shared memory; after that (and
// from then on) the normal matrix of the significant columns is formed in
// double-float and factored in FP64 in the CTA's global scratch slot, as the
// large path does near the optimum.  mnorm receives max_p M_pp.  Returns
// false if the FP64 factor meets a pivot that is not positive (M singular to
// working precision).
template <int T>
__device__ bool factor_lp(const BatchArgs& a, Ctx& c, bool& tier2, double* M64, double* dinv64, double& mnorm) {
  const int m = c.m, n = c.n;
  mnorm = 0.0;
  if (!tier2) {
    blk_syrk<T>(c, a.m_cap);
    double dm = 0.0;
    for (int i = threadIdx.x; i < m; i += T) dm = fmax(dm, (double)c.L[pk(i, i)]);
    mnorm = bmax<T>(dm, c.scal);
    tier2 = !blk_chol<T>(c);
  }
  if (!tier2) return true;
  // the significant columns: D_j >= 1e-10 max D, at least min(n, 1.25 m)
  // of them (the threshold drops by 16x until enough pass); the factor
  // of A_K D_K A_K' preconditions the exact M in the refinement
  double dmx = 0.0;
  for (int j = threadIdx.x; j < n; j += T) dmx = fmax(dmx, c.D[j]);
  dmx = bmax<T>(dmx, c.scal);
  const int want = min(n, (5 * m + 3) / 4);
  double thr = dmx * 1e-10;
  for (int guard = 0; guard < 64; ++guard) {
    int cnt = 0;
    for (int j = threadIdx.x; j < n; j += T) cnt += c.D[j] >= thr;
    if ((int)bsum<T>((double)cnt, c.scal) >= want) break;
    thr *= 0x1p-4;
  }
  if (threadIdx.x == 0) {  // ordered compaction
    int k = 0;
    for (int j = 0; j < n; ++j)
      if (c.D[j] >= thr) c.kidx[k++] = j;
    c.scal[31] = (double)k;
  }
  __syncthreads();
  const int nk = (int)c.scal[31];
  __syncthreads();
  blk_syrk_df<T>(c, a.m_cap, M64, nk);
  double dm = 0.0;
  for (int i = threadIdx.x; i < m; i += T) dm = fmax(dm, M64[pk(i, i)]);
  mnorm = bmax<T>(dm, c.scal);
  return blk_chol64<T>(c, M64, dinv64);
}

// out = (A D A')^{-1} rhs: out = P^-1 rhs, then preconditioned conjugate
// gradients on the exact M (matrix-free), accepted when ||rhs - M out||_inf
// <= refine_tol ||rhs||_inf or <= refine_tol (mnorm ||out||_inf +
// ||rhs||_inf).  Uses c.rho, c.z, c.p, c.q; leaves c.w = A' (last operand).
// Returns whether the tolerance was met within refine_max steps.
template <int T>
__device__ bool pcg_lp(const BatchArgs& a, Ctx& c, bool tier2, const double* M64, const double* dinv64,
                       double mnorm, const double* rhs, double* out, int refine_max) {
  const int m = c.m;
  double rn = 0.0;
  for (int i = threadIdx.x; i < m; i += T) rn = fmax(rn, fabs(rhs[i]));
  rn = bmax<T>(rn, c.scal);
  if (!(rn > 0.0)) rn = 1.0;
  auto precond = [&](const double* v, double* o) {
    if (tier2) blk_precond64<T>(c, M64, dinv64, v, o);
    else blk_precond<T>(c, v, o);
  };
  precond(rhs, out);
  auto accepted = [&](double res, double dyn) {
    return res <= a.refine_tol * rn || res <= a.refine_tol * (mnorm * dyn + rn);
  };
  auto true_residual = [&](double& res, double& dyn) {
    blk_apply_m<T>(c, out, rhs, c.rho);  // rho = rhs - M out
    double rr = 0.0, dd = 0.0;
    for (int i = threadIdx.x; i < m; i += T) {
      rr = fmax(rr, fabs(c.rho[i]));
      dd = fmax(dd, fabs(out[i]));
    }
    res = bmax<T>(rr, c.scal);
    dyn = bmax<T>(dd, c.scal);
  };
  double res, dyn;
  true_residual(res, dyn);
  bool done = accepted(res, dyn);
  if (!done) {
    double rz = 0.0;
    auto restart = [&]() {
      precond(c.rho, c.z);
      double t = 0.0;
      for (int i = threadIdx.x; i < m; i += T) {
        c.p[i] = c.z[i];
        t += c.rho[i] * c.z[i];
      }
      rz = bsum<T>(t, c.scal);
    };
    restart();
    for (int k = 0; k < refine_max && rz > 0.0 && isfinite(rz); ++k) {
      blk_apply_m<T>(c, c.p, nullptr, c.q, !tier2);
      double t = 0.0;
      for (int i = threadIdx.x; i < m; i += T) t += c.p[i] * c.q[i];
      const double pq = bsum<T>(t, c.scal);
      if (!(pq > 0.0)) break;
      const double al = rz / pq;
      double rr = 0.0, dd = 0.0;
      for (int i = threadIdx.x; i < m; i += T) {
        out[i] += al * c.p[i];
        c.rho[i] -= al * c.q[i];
        rr = fmax(rr, fabs(c.rho[i]));
        dd = fmax(dd, fabs(out[i]));
      }
      res = bmax<T>(rr, c.scal);
      dyn = bmax<T>(dd, c.scal);
      if (accepted(res, dyn) || k % 10 == 9) {
        true_residual(res, dyn);
        if ((done = accepted(res, dyn))) break;
        restart();
        continue;
      }
      precond(c.rho, c.z);
      t = 0.0;
      for (int i = threadIdx.x; i < m; i += T) t += c.rho[i] * c.z[i];
      const double rz2 = bsum<T>(t, c.scal);
      const double beta = rz2 / rz;
      for (int i = threadIdx.x; i < m; i += T) c.p[i] = c.z[i] + beta * c.p[i];
      __syncthreads();
      rz = rz2;
    }
  }
  return done;
}

// The whole PDAS loop of one LP; returns its status, iterations and gap.
template <int T>
__device__ void solve_lp(const BatchArgs& a, const BatchLP lp, Ctx& c, int& status, int& iters, double& gap,
                         int& n_shift, int& n_unref) {
  const int m = lp.m, n = lp.n;
  double* x = a.x + lp.n_off;
  double* s = a.s + lp.n_off;
  double* y = a.y + lp.m_off;
  const double* bv = a.b + lp.m_off;
  const double* cv = a.c + lp.n_off;
  status = PDAS_MAX_ITER;
  iters = 0;
  gap = NAN;
  n_shift = 0;
  n_unref = 0;
  int stalls = 0;
  bool tier2 = false;
  double* M64 = a.scratch + (int64_t)blockIdx.x * a.slot;
  double* dinv64 = M64 + (int64_t)a.m_cap * (a.m_cap + 1) / 2;
  for (int it = 0; it < a.max_iter; ++it) {
    // D = x / s and the interior check
    int bad = 0;
    for (int j = threadIdx.x; j < n; j += T) {
      const double xj = x[j], sj = s[j];
      if (!(xj > 0.0) || !(sj > 0.0) || !isfinite(xj) || !isfinite(sj)) bad = 1;
      c.D[j] = xj / sj;
      c.un2[j] = df_split(xj);
    }
    if (__syncthreads_or(bad)) {
      status = PDAS_ERR_NOT_INTERIOR;
      break;
    }
    blk_gemv<T>(c, c.un2, nullptr, c.r);  // r = A x
    __syncthreads();
    double mnorm = 0.0;
    // (a non-positive FP64 pivot means M is singular to working precision at
    // this iterate: a nearly degenerate LP close to its optimum)
    if (!factor_lp<T>(a, c, tier2, M64, dinv64, mnorm)) {
      status = PDAS_ERR_NOT_SPD;
      break;
    }
    if (tier2) ++n_shift;
    if (!pcg_lp<T>(a, c, tier2, M64, dinv64, mnorm, c.r, c.dy, a.refine_max)) ++n_unref;
    // w = A' dy; dx = D w - x; ds = -w
    blk_gemv_t<T>(c, c.dy, c.w);
    __syncthreads();
    double psi = -INFINITY;
    int nonfinite = 0;
    for (int j = threadIdx.x; j < n; j += T) {
      const double w = c.w[j], dx = c.D[j] * w - x[j];
      const double u = -dx / x[j], v = w / s[j];
      if (!isfinite(u) || !isfinite(v)) nonfinite = 1;
      psi = fmax(psi, fmax(u, v));
    }
    if (__syncthreads_or(nonfinite)) {
      status = PDAS_ERR_NONFINITE;
      break;
    }
    psi = bmax<T>(psi, c.scal);
    const double theta = psi <= 1.0 ? 1.0 : a.alpha / psi;
    double cx = 0.0, by = 0.0;
    for (int j = threadIdx.x; j < n; j += T) {
      const double w = c.w[j];
      const double xn = x[j] + theta * (c.D[j] * w - x[j]);
      x[j] = xn;
      s[j] = s[j] - theta * w;
      cx += cv[j] * xn;
    }
    for (int i = threadIdx.x; i < m; i += T) {
      const double yn = y[i] + theta * c.dy[i];
      y[i] = yn;
      by += bv[i] * yn;
    }
    cx = bsum<T>(cx, c.scal);
    by = bsum<T>(by, c.scal);
    gap = (cx - by) / (1.0 + fabs(cx));
    iters = it + 1;
    if (psi <= 1.0) {
      status = PDAS_OPTIMAL_EXACT;
      break;
    }
    if (gap < a.tol) {
      status = PDAS_OPTIMAL;
      break;
    }
    stalls = theta < 1e-12 ? stalls + 1 : 0;
    if (stalls >= 5) {
      status = PDAS_STALLED;
      break;
    }
  }
}

// The per-CTA views of the dynamic shared memory for capacities (m_cap, n_cap).
__device__ __forceinline__ Ctx make_ctx(unsigned char* batch_smem_raw, int m_cap, int n_cap) {
  const BatchSmem L = batch_smem(m_cap, n_cap);
  Ctx c;
  c.L = reinterpret_cast<float*>(batch_smem_raw + L.L);
  c.dinv = reinterpret_cast<float*>(batch_smem_raw + L.dinv);
  c.zf = reinterpret_cast<float*>(batch_smem_raw + L.zf);
  double* vm = reinterpret_cast<double*>(batch_smem_raw + L.vm);
  c.r = vm;
  c.dy = vm + m_cap;
  c.rho = vm + 2 * m_cap;
  c.z = vm + 3 * m_cap;
  c.p = vm + 4 * m_cap;
  c.q = vm + 5 * m_cap;
  c.D = reinterpret_cast<double*>(batch_smem_raw + L.D);
  c.w = reinterpret_cast<double*>(batch_smem_raw + L.w);
  c.un2 = reinterpret_cast<float2*>(batch_smem_raw + L.un2);
  c.pm2 = reinterpret_cast<float2*>(batch_smem_raw + L.pm2);
  c.kidx = reinterpret_cast<int*>(batch_smem_raw + L.kidx);
  c.stage = reinterpret_cast<float*>(batch_smem_raw + L.stage);
  c.dc = reinterpret_cast<float*>(batch_smem_raw + L.dc);
  c.scal = reinterpret_cast<double*>(batch_smem_raw + L.scal);
  return c;
}

template <int T>
__global__ void __launch_bounds__(T) k_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char batch_smem_raw[];
  __shared__ int s_lp;
  Ctx c = make_ctx(batch_smem_raw, a.m_cap, a.n_cap);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned t = atomicAdd(a.ticket, 1u);
      s_lp = t < (unsigned)a.count ? a.order[t] : -1;
    }
    __syncthreads();
    const int id = s_lp;
    if (id < 0) return;
    const BatchLP lp = a.lps[id];
    c.A = a.A + lp.a_off;
    c.m = lp.m;
    c.n = lp.n;
    int status, iters, n_shift, n_unref;
    double gap;
    uint64_t t0 = 0;
    if (threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    solve_lp<T>(a, lp, c, status, iters, gap, n_shift, n_unref);
    if (threadIdx.x == 0) {
      uint64_t t1;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
      a.time_us[id] = (float)((t1 - t0) * 1e-3);
      a.status[id] = status;
      a.iters[id] = iters;
      a.gap[id] = gap;
      a.shifted[id] = n_shift;
      a.unrefined[id] = n_unref;
    }
  }
}

// The adjoint of one LP at its final iterate (x, y, s), as pdas_backward
// (pdas.h) computes it for one handle: implicit differentiation of
// F = [A x - b; A'y + s - c; X s - sigma] = 0 with sigma = x.*s held fixed,
// whose adjoint system reduces to the normal equations of the direction,
//     (A D A') la = A D g,   lb = D (A' la - g),   lc = -lb / x,
// then two corrections on the full system J'(la, lb, lc) = (g, 0, 0) with
// FP64 residuals (lb alone cancels where D is large); each correction solves
// the same normal equations with right-hand side A (D r1 - r3 - lb).  M at
// the final D is formed and factored in the CTA (FP32 in shared memory, or
// the FP64 tier's factor if the FP32 one fails) and preconditions the
// conjugate gradients of every solve (at most 4 refine_max steps each).
// Outputs: dL/db = la, dL/dc = lb, dL/dA = -(la x' + y lb') (if wanted).
struct AdjointArgs {
  BatchArgs a;        // the solve's buffers: (x, y, s) hold the final iterates
  const double* g;    // dL/dx, packed like x
  double* la;         // dL/db, packed like y
  double* lb;         // dL/dc, packed like x
  double* dA;         // dL/dA, packed like A (FP64), or null
  double* lc;         // work, packed like x: multiplier of X s = sigma
  double* wt;         // work, packed like x: A' la
  double* r1;         // work, packed like x: residual of A' la + S lc = g
  double* r3;         // work, packed like x: residual of lb + X lc = 0
  int* astatus;       // per-LP status of the adjoint
};

template <int T>
__device__ int adjoint_lp(const AdjointArgs& g, const BatchLP lp, Ctx& c) {
  const BatchArgs& a = g.a;
  const int m = lp.m, n = lp.n;
  const double* x = a.x + lp.n_off;
  const double* s = a.s + lp.n_off;
  const double* y = a.y + lp.m_off;
  const double* gv = g.g + lp.n_off;
  double* la = g.la + lp.m_off;
  double* lb = g.lb + lp.n_off;
  double* lc = g.lc + lp.n_off;
  double* wt = g.wt + lp.n_off;
  double* r1 = g.r1 + lp.n_off;
  double* r3 = g.r3 + lp.n_off;
  double* M64 = a.scratch + (int64_t)blockIdx.x * a.slot;
  double* dinv64 = M64 + (int64_t)a.m_cap * (a.m_cap + 1) / 2;
  int bad = 0;
  for (int j = threadIdx.x; j < n; j += T) {
    const double xj = x[j], sj = s[j];
    if (!(xj > 0.0) || !(sj > 0.0) || !isfinite(xj) || !isfinite(sj)) bad = 1;
    c.D[j] = xj / sj;
    c.un2[j] = df_split(c.D[j] * gv[j]);  // D g
  }
  if (__syncthreads_or(bad)) return PDAS_ERR_NOT_INTERIOR;
  bool tier2 = false;
  double mnorm = 0.0;
  if (!factor_lp<T>(a, c, tier2, M64, dinv64, mnorm)) return PDAS_ERR_NOT_SPD;
  blk_gemv<T>(c, c.un2, nullptr, c.r);  // r = A D g
  __syncthreads();
  if (!pcg_lp<T>(a, c, tier2, M64, dinv64, mnorm, c.r, c.dy, 4 * a.refine_max)) return PDAS_ERR_NOT_SPD;
  for (int i = threadIdx.x; i < m; i += T) la[i] = c.dy[i];
  blk_gemv_t<T>(c, c.dy, c.w);  // A' la
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += T) {
    const double b = c.D[j] * (c.w[j] - gv[j]);
    lb[j] = b;
    lc[j] = -b / x[j];
    wt[j] = c.w[j];
  }
  __syncthreads();
  for (int it = 0; it < 2; ++it) {
    for (int j = threadIdx.x; j < n; j += T) {
      const double e1 = gv[j] - wt[j] - s[j] * lc[j];
      const double e3 = -lb[j] - x[j] * lc[j];
      r1[j] = e1;
      r3[j] = e3;
      c.un2[j] = df_split(c.D[j] * e1 - e3 - lb[j]);
    }
    __syncthreads();
    blk_gemv<T>(c, c.un2, nullptr, c.r);  // r = A (D r1 - r3 - lb)
    __syncthreads();
    // (no correction that meets the tolerance: it is at the rounding level; keep what we have)
    if (!pcg_lp<T>(a, c, tier2, M64, dinv64, mnorm, c.r, c.dy, 4 * a.refine_max)) break;
    for (int i = threadIdx.x; i < m; i += T) la[i] += c.dy[i];
    blk_gemv_t<T>(c, c.dy, c.w);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += T) {
      const double db = c.D[j] * (c.w[j] - r1[j]) + r3[j];
      lb[j] += db;
      lc[j] += (r3[j] - db) / x[j];
      wt[j] += c.w[j];
    }
    __syncthreads();
  }
  if (g.dA) {
    double* dA = g.dA + lp.a_off;
    for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += T) {
      const int p = (int)(e / n), j = (int)(e - (int64_t)p * n);
      dA[e] = -(la[p] * x[j] + y[p] * lb[j]);
    }
  }
  return PDAS_OK;
}

template <int T>
__global__ void __launch_bounds__(T) k_batch_adjoint(AdjointArgs g) {
  extern __shared__ __align__(16) unsigned char batch_smem_raw[];
  __shared__ int s_lp;
  const BatchArgs& a = g.a;
  Ctx c = make_ctx(batch_smem_raw, a.m_cap, a.n_cap);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned t = atomicAdd(a.ticket, 1u);
      s_lp = t < (unsigned)a.count ? a.order[t] : -1;
    }
    __syncthreads();
    const int id = s_lp;
    if (id < 0) return;
    const BatchLP lp = a.lps[id];
    c.A = a.A + lp.a_off;
    c.m = lp.m;
    c.n = lp.n;
    const int st = adjoint_lp<T>(g, lp, c);
    if (threadIdx.x == 0) g.astatus[id] = st;
  }
}

// ---------------------------------------------------------------------------
constexpr int kBuckets = 4;  // m in [1, 64], (64, 128], (128, 192], (192, 256]
constexpr int kCandidates[3] = {128, 256, 512};

cudaError_t set_smem_attr(int threads, size_t bytes) {
  if (threads == 128) return cudaFuncSetAttribute(k_batch<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (threads == 256) return cudaFuncSetAttribute(k_batch<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaFuncSetAttribute(k_batch<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
cudaError_t occupancy(int threads, size_t bytes, int* blocks) {
  if (threads == 128) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_batch<128>, 128, bytes);
  if (threads == 256) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_batch<256>, 256, bytes);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_batch<512>, 512, bytes);
}
cudaError_t launch(int threads, int grid, size_t bytes, cudaStream_t st, const BatchArgs& a) {
  if (threads == 128) k_batch<128><<<grid, 128, bytes, st>>>(a);
  else if (threads == 256) k_batch<256><<<grid, 256, bytes, st>>>(a);
  else k_batch<512><<<grid, 512, bytes, st>>>(a);
  return cudaGetLastError();
}
// The adjoint kernel of a bucket uses the solve kernel's shared-memory layout
// and CTA size; its grid comes from its own occupancy.
cudaError_t set_adjoint_smem_attr(int threads, size_t bytes) {
  if (threads == 128)
    return cudaFuncSetAttribute(k_batch_adjoint<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (threads == 256)
    return cudaFuncSetAttribute(k_batch_adjoint<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaFuncSetAttribute(k_batch_adjoint<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
cudaError_t adjoint_occupancy(int threads, size_t bytes, int* blocks) {
  if (threads == 128) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_batch_adjoint<128>, 128, bytes);
  if (threads == 256) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_batch_adjoint<256>, 256, bytes);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_batch_adjoint<512>, 512, bytes);
}
cudaError_t launch_adjoint(int threads, int grid, size_t bytes, cudaStream_t st, const AdjointArgs& g) {
  if (threads == 128) k_batch_adjoint<128><<<grid, 128, bytes, st>>>(g);
  else if (threads == 256) k_batch_adjoint<256><<<grid, 256, bytes, st>>>(g);
  else k_batch_adjoint<512><<<grid, 512, bytes, st>>>(g);
  return cudaGetLastError();
}

}  // namespace
}  // namespace pdas

using namespace pdas;

struct pdas_batch_ctx {
  pdas_batch_options opt{};
  cudaStream_t st = nullptr;
  bool own_stream = false;  // (no stream given: graphs cannot be captured on the legacy stream)
  int count = 0;
  int sms = 0;
  const float* A = nullptr;
  const double *b = nullptr, *c = nullptr;
  double *x = nullptr, *y = nullptr, *s = nullptr;
  BatchLP* lps = nullptr;  // device
  int* order = nullptr;    // device, bucket after bucket
  int* status = nullptr;   // device outputs
  int* iters = nullptr;
  double* gap = nullptr;
  int* shifted = nullptr;
  int* unrefined = nullptr;
  float* time_us = nullptr;
  unsigned* tickets = nullptr;  // one per bucket
  double* scratch = nullptr;    // FP64 tier slots, one per LP of each bucket
  int64_t total_m = 0, total_n = 0;
  double* adj_work = nullptr;   // the adjoint's four n-packed work vectors
  int* astatus = nullptr;       // per-LP status of the last adjoint (device)
  int* h_astatus = nullptr;     // (pinned mirror)
  int* h_status = nullptr;      // pinned mirrors
  int* h_iters = nullptr;
  double* h_gap = nullptr;
  int* h_shifted = nullptr;
  int* h_unrefined = nullptr;
  float* h_time_us = nullptr;
  struct Bucket {
    int m_bound = 0, m_cap = 0, n_cap = 0, count = 0, offset = 0, threads = 256, grid = 0, adj_grid = 0;
    int64_t slot = 0, scratch_off = 0;  // doubles per FP64-tier slot; first slot of the bucket
    size_t smem = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t done = nullptr;
  } bk[kBuckets];
  cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double last_ms = -1.0;
  char errmsg[256] = {0};
};

namespace {

pdas_status cuda_fail(pdas_batch_ctx* h, cudaError_t e, const char* where) {
  snprintf(h->errmsg, sizeof(h->errmsg), "%s: %s", where, cudaGetErrorString(e));
  return PDAS_ERR_CUDA;
}

#define BCK(call)                                         \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

BatchArgs bucket_args(const pdas_batch_ctx* h, int bi, double* x, double* y, double* s, int max_iter) {
  const auto& B = h->bk[bi];
  BatchArgs a;
  a.lps = h->lps;
  a.order = h->order + B.offset;
  a.count = B.count;
  a.m_cap = B.m_cap;
  a.n_cap = B.n_cap;
  a.A = h->A;
  a.b = h->b;
  a.c = h->c;
  a.x = x;
  a.y = y;
  a.s = s;
  a.alpha = h->opt.alpha;
  a.tol = h->opt.tol;
  a.refine_tol = h->opt.refine_tol;
  a.max_iter = max_iter;
  a.refine_max = h->opt.refine_max;
  a.status = h->status;
  a.iters = h->iters;
  a.gap = h->gap;
  a.shifted = h->shifted;
  a.unrefined = h->unrefined;
  a.time_us = h->time_us;
  a.ticket = h->tickets + bi;
  a.scratch = h->scratch + B.scratch_off;
  a.slot = B.slot;
  return a;
}

pdas_status grid_for_bucket(pdas_batch_ctx* h, int bi, int threads, int* grid) {
  auto& B = h->bk[bi];
  int occ = 0;
  BCK(set_smem_attr(threads, B.smem));
  BCK(occupancy(threads, B.smem, &occ));
  if (occ < 1) return PDAS_ERR_UNSUPPORTED;
  *grid = std::min(B.count, occ * h->sms);
  return PDAS_OK;
}

// Times each candidate CTA size on two iterations of every LP of the bucket,
// run on scratch copies of (x, y, s), and keeps the fastest.
pdas_status autotune(pdas_batch_ctx* h, int64_t nx, int64_t ny) {
  double *sx = nullptr, *sy = nullptr, *ss = nullptr;
  cudaError_t e = cudaMalloc(&sx, sizeof(double) * nx);
  if (e == cudaSuccess) e = cudaMalloc(&sy, sizeof(double) * ny);
  if (e == cudaSuccess) e = cudaMalloc(&ss, sizeof(double) * nx);
  pdas_status st = PDAS_OK;
  for (int bi = 0; bi < kBuckets && e == cudaSuccess && st == PDAS_OK; ++bi) {
    auto& B = h->bk[bi];
    if (B.count == 0) continue;
    float best = INFINITY;
    for (int threads : kCandidates) {
      int grid = 0;
      if (grid_for_bucket(h, bi, threads, &grid) != PDAS_OK) {
        cudaGetLastError();
        continue;
      }
      float ms_min = INFINITY;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        e = cudaMemcpyAsync(sx, h->x, sizeof(double) * nx, cudaMemcpyDeviceToDevice, h->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sy, h->y, sizeof(double) * ny, cudaMemcpyDeviceToDevice, h->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ss, h->s, sizeof(double) * nx, cudaMemcpyDeviceToDevice, h->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->tickets + bi, 0, sizeof(unsigned), h->st);
        if (e == cudaSuccess) e = cudaEventRecord(h->t0, h->st);
        if (e == cudaSuccess) e = launch(threads, grid, B.smem, h->st, bucket_args(h, bi, sx, sy, ss, 2));
        if (e == cudaSuccess) e = cudaEventRecord(h->t1, h->st);
        if (e == cudaSuccess) e = cudaEventSynchronize(h->t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, h->t0, h->t1);
        if (e == cudaSuccess) ms_min = std::min(ms_min, ms);
      }
      if (e == cudaSuccess && ms_min < best) {
        best = ms_min;
        B.threads = threads;
        B.grid = grid;
      }
    }
    if (!(best < INFINITY)) st = PDAS_ERR_UNSUPPORTED;
  }
  if (sx) cudaFree(sx);
  if (sy) cudaFree(sy);
  if (ss) cudaFree(ss);
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
  return st;
}

// One graph: reset the queues, fork one branch per non-empty bucket (its
// persistent launch on a side stream), join, copy the per-LP results to the
// pinned host mirrors.
pdas_status capture(pdas_batch_ctx* h) {
  BCK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemsetAsync(h->tickets, 0, sizeof(unsigned) * kBuckets, h->st);
  if (e == cudaSuccess) e = cudaEventRecord(h->fork, h->st);
  for (int bi = 0; bi < kBuckets && e == cudaSuccess; ++bi) {
    auto& B = h->bk[bi];
    if (B.count == 0) continue;
    e = cudaStreamWaitEvent(B.side, h->fork, 0);
    if (e == cudaSuccess) e = launch(B.threads, B.grid, B.smem, B.side, bucket_args(h, bi, h->x, h->y, h->s, h->opt.max_iter));
    if (e == cudaSuccess) e = cudaEventRecord(B.done, B.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->st, B.done, 0);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_status, h->status, sizeof(int) * h->count, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_iters, h->iters, sizeof(int) * h->count, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_gap, h->gap, sizeof(double) * h->count, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_shifted, h->shifted, sizeof(int) * h->count, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_unrefined, h->unrefined, sizeof(int) * h->count, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_time_us, h->time_us, sizeof(float) * h->count, cudaMemcpyDeviceToHost, h->st);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(h->st, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(h, e, "capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
  h->graph = g;
  BCK(cudaGraphInstantiate(&h->exec, h->graph, 0));
  return PDAS_OK;
}

}  // namespace

extern "C" {

void pdas_batch_default_options(pdas_batch_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->alpha = 0.95;
  opt->tol = 1e-7;
  opt->max_iter = 500;
  opt->refine_tol = 1e-14;
  opt->refine_max = 40;
  opt->autotune = 1;
  opt->stream = nullptr;
}

void pdas_batch_destroy(pdas_batch_handle h) {
  if (!h) return;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  for (auto& B : h->bk) {
    if (B.side) cudaStreamDestroy(B.side);
    if (B.done) cudaEventDestroy(B.done);
  }
  if (h->fork) cudaEventDestroy(h->fork);
  if (h->t0) cudaEventDestroy(h->t0);
  if (h->t1) cudaEventDestroy(h->t1);
  if (h->own_stream && h->st) cudaStreamDestroy(h->st);
  if (h->lps) cudaFree(h->lps);
  if (h->order) cudaFree(h->order);
  if (h->status) cudaFree(h->status);
  if (h->iters) cudaFree(h->iters);
  if (h->gap) cudaFree(h->gap);
  if (h->shifted) cudaFree(h->shifted);
  if (h->unrefined) cudaFree(h->unrefined);
  if (h->h_shifted) cudaFreeHost(h->h_shifted);
  if (h->h_unrefined) cudaFreeHost(h->h_unrefined);
  if (h->time_us) cudaFree(h->time_us);
  if (h->h_time_us) cudaFreeHost(h->h_time_us);
  if (h->tickets) cudaFree(h->tickets);
  if (h->scratch) cudaFree(h->scratch);
  if (h->h_status) cudaFreeHost(h->h_status);
  if (h->adj_work) cudaFree(h->adj_work);
  if (h->astatus) cudaFree(h->astatus);
  if (h->h_astatus) cudaFreeHost(h->h_astatus);
  if (h->h_iters) cudaFreeHost(h->h_iters);
  if (h->h_gap) cudaFreeHost(h->h_gap);
  delete h;
}

pdas_status pdas_batch_create(int count, const int* m, const int* n, const float* A, const double* b,
                              const double* c, double* x, double* y, double* s, const pdas_batch_options* opt_in,
                              pdas_batch_handle* out) {
  if (!out) return PDAS_ERR_ARG;
  *out = nullptr;
  if (count < 1 || !m || !n || !A || !b || !c || !x || !y || !s) return PDAS_ERR_ARG;
  pdas_batch_options opt;
  if (opt_in) opt = *opt_in;
  else pdas_batch_default_options(&opt);
  if (!(opt.alpha > 0.0 && opt.alpha < 1.0) || !(opt.tol > 0.0) || opt.max_iter < 1 || !(opt.refine_tol >= 0.0) ||
      opt.refine_max < 0 || (opt.autotune & ~1))
    return PDAS_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (m[i] < 1 || n[i] <= m[i] || m[i] > PDAS_BATCH_MAX_M || n[i] > PDAS_BATCH_MAX_N) return PDAS_ERR_ARG;
  for (const void* p : {(const void*)A, (const void*)b, (const void*)c, (const void*)x, (const void*)y, (const void*)s})
    if ((uintptr_t)p % 16) return PDAS_ERR_ARG;
  pdas_batch_ctx* h = new (std::nothrow) pdas_batch_ctx();
  if (!h) return PDAS_ERR_CUDA;
  h->opt = opt;
  h->st = (cudaStream_t)opt.stream;
  h->count = count;
  h->A = A;
  h->b = b;
  h->c = c;
  h->x = x;
  h->y = y;
  h->s = s;
  // LP table and buckets (largest m * n first within a bucket)
  std::vector<BatchLP> lps(count);
  int64_t ao = 0, mo = 0, no = 0;
  for (int i = 0; i < count; ++i) {
    lps[i] = BatchLP{m[i], n[i], ao, mo, no};
    ao += (int64_t)m[i] * n[i];
    mo += m[i];
    no += n[i];
  }
  std::vector<int> order;
  order.reserve(count);
  for (int bi = 0; bi < kBuckets; ++bi) {
    auto& B = h->bk[bi];
    B.m_bound = 64 * (bi + 1);
    B.offset = (int)order.size();
    std::vector<int> ids;
    int nmax = 0;
    for (int i = 0; i < count; ++i)
      if (m[i] > B.m_bound - 64 && m[i] <= B.m_bound) {
        ids.push_back(i);
        nmax = std::max(nmax, n[i]);
      }
    std::stable_sort(ids.begin(), ids.end(), [&](int p, int q) {
      return (int64_t)m[p] * n[p] > (int64_t)m[q] * n[q];
    });
    B.count = (int)ids.size();
    B.m_cap = B.m_bound;
    B.n_cap = (nmax + 31) / 32 * 32;
    B.smem = batch_smem(B.m_cap, std::max(B.n_cap, 32)).total;
    B.slot = (int64_t)B.m_cap * (B.m_cap + 1) / 2 + B.m_cap;
    order.insert(order.end(), ids.begin(), ids.end());
  }
  int64_t scratch_total = 0;  // a launch's grid never exceeds its bucket's LP count
  for (auto& B : h->bk) {
    B.scratch_off = scratch_total;
    scratch_total += B.slot * B.count;
  }
  pdas_status st = PDAS_OK;
  auto fail = [&](pdas_status code) {
    pdas_batch_destroy(h);
    return code;
  };
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && !h->st) {
    e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
    h->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaMalloc(&h->lps, sizeof(BatchLP) * count);
  if (e == cudaSuccess) e = cudaMalloc(&h->order, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMalloc(&h->status, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMalloc(&h->iters, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMalloc(&h->gap, sizeof(double) * count);
  if (e == cudaSuccess) e = cudaMalloc(&h->shifted, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMalloc(&h->unrefined, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_shifted, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_unrefined, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMalloc(&h->time_us, sizeof(float) * count);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_time_us, sizeof(float) * count);
  if (e == cudaSuccess) e = cudaMalloc(&h->tickets, sizeof(unsigned) * kBuckets);
  if (e == cudaSuccess) e = cudaMalloc(&h->scratch, sizeof(double) * std::max<int64_t>(scratch_total, 1));
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_status, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_iters, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_gap, sizeof(double) * count);
  h->total_m = mo;
  h->total_n = no;
  if (e == cudaSuccess) e = cudaMalloc(&h->adj_work, sizeof(double) * 4 * no);
  if (e == cudaSuccess) e = cudaMalloc(&h->astatus, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_astatus, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMemcpy(h->lps, lps.data(), sizeof(BatchLP) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&h->t0);
  if (e == cudaSuccess) e = cudaEventCreate(&h->t1);
  for (auto& B : h->bk) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B.side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B.done, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    cuda_fail(h, e, "pdas_batch_create");
    return fail(PDAS_ERR_CUDA);
  }
  // CTA sizes: built-in choice (256), or the autotuner's
  for (int bi = 0; bi < kBuckets; ++bi) {
    auto& B = h->bk[bi];
    if (B.count == 0) continue;
    B.threads = 256;
    if ((st = grid_for_bucket(h, bi, B.threads, &B.grid)) != PDAS_OK) return fail(st);
  }
  if (opt.autotune && (st = autotune(h, no, mo)) != PDAS_OK) return fail(st);
  for (int bi = 0; bi < kBuckets; ++bi) {  // (the attribute is per function: set it for the final choice)
    auto& B = h->bk[bi];
    if (B.count && (st = grid_for_bucket(h, bi, B.threads, &B.grid)) != PDAS_OK) return fail(st);
    if (B.count) {  // the adjoint kernel of the bucket: same CTA size and shared memory
      int occ = 0;
      e = set_adjoint_smem_attr(B.threads, B.smem);
      if (e == cudaSuccess) e = adjoint_occupancy(B.threads, B.smem, &occ);
      if (e != cudaSuccess) {
        cuda_fail(h, e, "adjoint kernel attributes");
        return fail(PDAS_ERR_CUDA);
      }
      if (occ < 1) return fail(PDAS_ERR_UNSUPPORTED);
      B.adj_grid = std::min(B.count, occ * h->sms);
    }
  }
  if ((st = capture(h)) != PDAS_OK) return fail(st);
  *out = h;
  return PDAS_OK;
}

pdas_status pdas_batch_solve(pdas_batch_handle h, int* status_out, int* iters_out, double* gap_out) {
  if (!h) return PDAS_ERR_ARG;
  BCK(cudaEventRecord(h->t0, h->st));
  BCK(cudaGraphLaunch(h->exec, h->st));
  BCK(cudaEventRecord(h->t1, h->st));
  BCK(cudaStreamSynchronize(h->st));
  float ms = 0.f;
  BCK(cudaEventElapsedTime(&ms, h->t0, h->t1));
  h->last_ms = ms;
  if (status_out) memcpy(status_out, h->h_status, sizeof(int) * h->count);
  if (iters_out) memcpy(iters_out, h->h_iters, sizeof(int) * h->count);
  if (gap_out) memcpy(gap_out, h->h_gap, sizeof(double) * h->count);
  return PDAS_OK;
}

int pdas_batch_config(pdas_batch_handle h, int* m_bound, int* threads, int* lp_count, int cap) {
  if (!h) return 0;
  int k = 0;
  for (int bi = 0; bi < kBuckets; ++bi) {
    if (k < cap) {
      if (m_bound) m_bound[k] = h->bk[bi].m_bound;
      if (threads) threads[k] = h->bk[bi].threads;
      if (lp_count) lp_count[k] = h->bk[bi].count;
    }
    ++k;
  }
  return k;
}

double pdas_batch_last_ms(pdas_batch_handle h) { return h ? h->last_ms : -1.0; }

pdas_status pdas_batch_diagnostics(pdas_batch_handle h, int* fp64_out, int* unrefined_out, float* time_us_out) {
  if (!h) return PDAS_ERR_ARG;
  if (fp64_out) memcpy(fp64_out, h->h_shifted, sizeof(int) * h->count);
  if (unrefined_out) memcpy(unrefined_out, h->h_unrefined, sizeof(int) * h->count);
  if (time_us_out) memcpy(time_us_out, h->h_time_us, sizeof(float) * h->count);
  return PDAS_OK;
}

const char* pdas_batch_last_error_message(pdas_batch_handle h) { return h ? h->errmsg : ""; }

pdas_status pdas_batch_backward(pdas_batch_handle h, const double* dL_dx, double* dL_dA, double* dL_db,
                                double* dL_dc, int* status_out) {
  if (!h || !dL_dx || !dL_db || !dL_dc) return PDAS_ERR_ARG;
  for (const void* p : {(const void*)dL_dx, (const void*)dL_dA, (const void*)dL_db, (const void*)dL_dc})
    if ((uintptr_t)p % 16) return PDAS_ERR_ARG;
  BCK(cudaMemsetAsync(h->tickets, 0, sizeof(unsigned) * kBuckets, h->st));
  for (int bi = 0; bi < kBuckets; ++bi) {
    const auto& B = h->bk[bi];
    if (B.count == 0) continue;
    AdjointArgs g;
    g.a = bucket_args(h, bi, h->x, h->y, h->s, h->opt.max_iter);
    g.g = dL_dx;
    g.la = dL_db;
    g.lb = dL_dc;
    g.dA = dL_dA;
    g.lc = h->adj_work;
    g.wt = h->adj_work + h->total_n;
    g.r1 = h->adj_work + 2 * h->total_n;
    g.r3 = h->adj_work + 3 * h->total_n;
    g.astatus = h->astatus;
    BCK(launch_adjoint(B.threads, B.adj_grid, B.smem, h->st, g));
  }
  BCK(cudaMemcpyAsync(h->h_astatus, h->astatus, sizeof(int) * h->count, cudaMemcpyDeviceToHost, h->st));
  BCK(cudaStreamSynchronize(h->st));
  if (status_out) memcpy(status_out, h->h_astatus, sizeof(int) * h->count);
  return PDAS_OK;
}

}  // extern "C"
