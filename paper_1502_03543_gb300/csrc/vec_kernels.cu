// vec_kernels.cu -- the bandwidth-bound steps of one PDAS iteration:
//   scaling D = S^{-1} X (Eq. 4), the right-hand side r = A x and the
//   refinement residual r - A(D(A' dy)) (Section V), the direction
//   ds = -A' dy, dx = D(-ds) - x (Section V), the psi ratio test and the step
//   (algorithm of Section III).
//
// All sums are deterministic: every thread accumulates a fixed strided slice,
// blocks reduce with a fixed shuffle tree, and the last block to finish
// (ticket counter, no float atomics) combines the per-block partials in block
// order.  The grid of each reduction depends on the sizes only, so results
// are bit-identical from run to run.
#include "reduce_util.cuh"

namespace pdas {

namespace {

// ---- vector loads of VEC consecutive elements of A, widened to double ----
template <typename T>
struct Vec;
template <>
struct Vec<double> {
  static constexpr int N = 2;
  __device__ static void load(const double* p, double* o) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = v.x; o[1] = v.y;
  }
};
template <>
struct Vec<float> {
  static constexpr int N = 4;
  __device__ static void load(const float* p, double* o) {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    o[0] = widen_bits(v.x); o[1] = widen_bits(v.y); o[2] = widen_bits(v.z); o[3] = widen_bits(v.w);
  }
};
template <>
struct Vec<__nv_bfloat16> {
  static constexpr int N = 8;
  __device__ static void load(const __nv_bfloat16* p, double* o) {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[2 * i] = widen_bits(w[i] << 16);
      o[2 * i + 1] = widen_bits(w[i] & 0xffff0000u);
    }
  }
};

// ---------------------------------------------------------------------------
// a1: D = x/s, with max/min of D and the interior check.
__global__ void __launch_bounds__(kThreads) k_scaling(int64_t n, const double* __restrict__ x,
                                                      const double* __restrict__ s, double* __restrict__ D,
                                                      double* part, unsigned* tickets, Scalars* sc) {
  __shared__ double sm[32];
  double mx = -INFINITY, mn = INFINITY;
  int bad = 0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double xj = x[j], sj = s[j];
    if (!(xj > 0.0) || !(sj > 0.0) || !isfinite(xj) || !isfinite(sj)) bad = 1;
    const double d = xj / sj;
    D[j] = d;
    mx = fmax(mx, d);
    mn = fmin(mn, d);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&sc->bad_iterate, 1);
  double bmx = block_reduce<1>(mx, sm);
  double bmn = block_reduce<2>(mn, sm);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = bmx;
    part[2 * blockIdx.x + 1] = bmn;
  }
  if (!last_block(tickets + T_SCALING)) return;
  double gmx = -INFINITY, gmn = INFINITY;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    gmx = fmax(gmx, __ldcg(part + 2 * i));
    gmn = fmin(gmn, __ldcg(part + 2 * i + 1));
  }
  gmx = block_reduce<1>(gmx, sm);
  gmn = block_reduce<2>(gmn, sm);
  if (threadIdx.x == 0) {
    sc->dmax = gmx;
    sc->dmin = gmn;
    if (sc->bad_iterate && sc->status == 0) sc->status = PDAS_ERR_NOT_INTERIOR;
    tickets[T_SCALING] = 0;
  }
}

// ---------------------------------------------------------------------------
// a2 / a6: out_p = A_p. v  (base == null)  or  out_p = base_p - A_p. v.
// ROWS rows per block; FP64 accumulation of exactly widened A.  With
// norm_slot >= 0 also reduces max_p |out_p| into sc->rnorm (slot 0) or
// sc->rho_norm (slot 1).
template <typename T, int ROWS>
__global__ void __launch_bounds__(kThreads) k_gemv(int64_t m, int64_t n, const T* __restrict__ A,
                                                   const double* __restrict__ v, const double* __restrict__ base,
                                                   double* __restrict__ out, int vec_ok, double* part,
                                                   unsigned* tickets, Scalars* sc, int norm_slot) {
  __shared__ double sm[32];
  __shared__ double rowsum[ROWS];
  if (failed(sc)) return;
  constexpr int VN = Vec<T>::N;
  const int64_t p0 = (int64_t)blockIdx.x * ROWS;
  double acc[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) acc[r] = 0.0;
  if (vec_ok) {
    for (int64_t j = (int64_t)threadIdx.x * VN; j < n; j += (int64_t)blockDim.x * VN) {
      double vv[VN];
#pragma unroll
      for (int k = 0; k < VN; ++k) vv[k] = __ldg(v + j + k);
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        if (p0 + r < m) {
          double a[VN];
          Vec<T>::load(A + (p0 + r) * n + j, a);
#pragma unroll
          for (int k = 0; k < VN; ++k) acc[r] = fma(a[k], vv[k], acc[r]);
        }
      }
    }
  } else {
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const double vj = __ldg(v + j);
#pragma unroll
      for (int r = 0; r < ROWS; ++r)
        if (p0 + r < m) acc[r] = fma(widen(A[(p0 + r) * n + j]), vj, acc[r]);
    }
  }
  double amax = 0.0;
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    double t = block_reduce<0>(acc[r], sm);
    if (threadIdx.x == 0) rowsum[r] = t;
  }
  __syncthreads();
  if (threadIdx.x < ROWS && p0 + threadIdx.x < m) {
    const int64_t p = p0 + threadIdx.x;
    const double o = base ? base[p] - rowsum[threadIdx.x] : rowsum[threadIdx.x];
    out[p] = o;
    amax = fabs(o);
    if (!isfinite(o)) amax = INFINITY;
  }
  if (norm_slot < 0) return;
  double bm = block_reduce<1>(amax, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = bm;
  if (!last_block(tickets + T_NORM)) return;
  double g = combine<1>(part, gridDim.x, sm);
  if (threadIdx.x == 0) {
    if (norm_slot == 0) sc->rnorm = g; else sc->rho_norm = g;
    tickets[T_NORM] = 0;
  }
}

// ---------------------------------------------------------------------------
// a7 (first half): partial column sums part[c][j] = sum_{p in chunk c} A_pj u_p.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_gemv_t_part(int64_t m, int64_t n, const T* __restrict__ A,
                                                          const double* __restrict__ u, double* __restrict__ part,
                                                          int64_t rows_per_chunk, int vec_ok) {
  constexpr int VN = Vec<T>::N;
  const int64_t pbeg = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t pend = pbeg + rows_per_chunk < m ? pbeg + rows_per_chunk : m;
  double* dst = part + (int64_t)blockIdx.y * n;
  if (vec_ok) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VN;
    if (j >= n) return;
    double acc[VN];
#pragma unroll
    for (int k = 0; k < VN; ++k) acc[k] = 0.0;
    for (int64_t p = pbeg; p < pend; ++p) {
      double a[VN];
      Vec<T>::load(A + p * n + j, a);
      const double up = __ldg(u + p);
#pragma unroll
      for (int k = 0; k < VN; ++k) acc[k] = fma(a[k], up, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < VN; ++k) dst[j + k] = acc[k];
  } else {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double acc = 0.0;
    for (int64_t p = pbeg; p < pend; ++p) acc = fma(widen(A[p * n + j]), __ldg(u + p), acc);
    dst[j] = acc;
  }
}

// a7 (second half): w_j = sum_c part[c][j] in chunk order, then the mode's
// elementwise outputs.
__global__ void __launch_bounds__(kThreads) k_gemv_t_finish(int64_t n, int chunks, const double* __restrict__ part,
                                                            int mode, const double* __restrict__ x,
                                                            const double* __restrict__ D, double* out0,
                                                            double* out1, double* out2, const Scalars* sc,
                                                            const double* __restrict__ rd) {
  if (failed(sc)) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double w = 0.0;
    if (mode == 3) w = out2[j];
    else
      for (int c = 0; c < chunks; ++c) w += __ldcg(part + (int64_t)c * n + j);
    if (mode == 0) {
      out0[j] = w;
    } else if (mode == 1 || mode == 3) {
      const double ds = rd ? rd[j] - w : -w;
      out0[j] = D[j] * (-ds) - x[j];  // dx = D(-ds) - x
      out1[j] = ds;
      if (out2 && mode == 1) out2[j] = w;
    } else {
      out0[j] = D[j] * w;
      if (out2) out2[j] = w;
    }
  }
}

// Infeasible-start variant: the dual residual rd = c - A'y - s (w = A'y) of
// the second row of Eq. (3), and nu = -(D rd) for the right-hand side
// b - A nu = b + A D rd of the normal equations.
__global__ void k_dual_residual(int64_t n, const double* __restrict__ c, const double* __restrict__ s,
                                const double* __restrict__ w, const double* __restrict__ D, double* __restrict__ rd,
                                double* __restrict__ nu, const Scalars* sc) {
  if (failed(sc)) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double r = (c[j] - w[j]) - s[j];
    rd[j] = r;
    nu[j] = -(D[j] * r);
  }
}

// Relative residuals of the iterate: max|rp| / (1 + max|b|) and
// max|(c - w) - s| / (1 + max|c|), four maxima per block, combined in block
// order by the last block.  NaN propagates as Inf.
__global__ void __launch_bounds__(kThreads) k_residual_norms(int64_t m, int64_t n, const double* __restrict__ b,
                                                             const double* __restrict__ rp,
                                                             const double* __restrict__ c,
                                                             const double* __restrict__ w,
                                                             const double* __restrict__ s, double* part,
                                                             unsigned* tickets, Scalars* sc) {
  __shared__ double sm[32];
  if (failed(sc)) return;
  double v[4] = {0.0, 0.0, 0.0, 0.0};  // |rp|, |b|, |rd|, |c|
  auto upd = [](double& acc, double a) { acc = (a == a) ? fmax(acc, fabs(a)) : INFINITY; };
  const int64_t len = n > m ? n : m;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x) {
    if (j < m) {
      upd(v[0], rp[j]);
      upd(v[1], b[j]);
    }
    if (j < n) {
      upd(v[2], (c[j] - w[j]) - s[j]);
      upd(v[3], c[j]);
    }
  }
  for (int k = 0; k < 4; ++k) {
    const double r = block_reduce<1>(v[k], sm);
    if (threadIdx.x == 0) part[4 * blockIdx.x + k] = r;
  }
  if (!last_block(tickets + T_RES)) return;
  if (threadIdx.x == 0) {
    double g[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < (int)gridDim.x; ++i)
      for (int k = 0; k < 4; ++k) g[k] = fmax(g[k], __ldcg(part + 4 * i + k));
    sc->pres = g[0] / (1.0 + g[1]);
    sc->dres = g[2] / (1.0 + g[3]);
    tickets[T_RES] = 0;
  }
}

// ---------------------------------------------------------------------------
// a8: psi = max_j max(-dx_j/x_j, -ds_j/s_j); theta = alpha/psi, or 1 if psi <= 1
// (capped, the infeasible-start variant: min(1, alpha/psi)).
__global__ void __launch_bounds__(kThreads) k_psi(int64_t n, const double* __restrict__ x,
                                                  const double* __restrict__ s, const double* __restrict__ dx,
                                                  const double* __restrict__ ds, double alpha, double* part,
                                                  unsigned* tickets, Scalars* sc, int capped) {
  __shared__ double sm[32];
  if (failed(sc)) return;
  double mx = -INFINITY;
  int bad = 0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double u = -dx[j] / x[j];
    const double v = -ds[j] / s[j];
    if (!isfinite(u) || !isfinite(v)) bad = 1;
    mx = fmax(mx, fmax(u, v));
  }
  bad = __syncthreads_or(bad);
  double bm = block_reduce<1>(mx, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = bad ? NAN : bm;
  if (!last_block(tickets + T_PSI)) return;
  double g = -INFINITY;
  int gbad = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    const double p = __ldcg(part + i);
    if (p != p) gbad = 1;
    g = fmax(g, p);
  }
  gbad = __syncthreads_or(gbad);
  g = block_reduce<1>(g, sm);
  if (threadIdx.x == 0) {
    sc->psi = g;
    sc->theta = capped ? (g <= alpha ? 1.0 : alpha / g) : (g <= 1.0 ? 1.0 : alpha / g);
    if (gbad) sc->status = PDAS_ERR_NONFINITE;
    tickets[T_PSI] = 0;
  }
}

// a9: (x,y,s) += theta (dx,dy,ds); then c'x, b'y, x's and the relative gap.
__global__ void __launch_bounds__(kThreads) k_step(int64_t m, int64_t n, const double* __restrict__ b,
                                                   const double* __restrict__ c, double* x, double* y, double* s,
                                                   const double* __restrict__ dx, const double* __restrict__ dy,
                                                   const double* __restrict__ ds, double* part, unsigned* tickets,
                                                   Scalars* sc) {
  __shared__ double sm[32];
  if (failed(sc)) return;
  const double th = sc->theta;
  double cx = 0.0, by = 0.0, xs = 0.0;
  const int64_t len = n > m ? n : m;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x) {
    if (j < n) {
      const double xn = x[j] + th * dx[j];
      const double sn = s[j] + th * ds[j];
      x[j] = xn;
      s[j] = sn;
      cx = fma(c[j], xn, cx);
      xs = fma(xn, sn, xs);
    }
    if (j < m) {
      const double yn = y[j] + th * dy[j];
      y[j] = yn;
      by = fma(b[j], yn, by);
    }
  }
  cx = block_reduce<0>(cx, sm);
  by = block_reduce<0>(by, sm);
  xs = block_reduce<0>(xs, sm);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = cx;
    part[3 * blockIdx.x + 1] = by;
    part[3 * blockIdx.x + 2] = xs;
  }
  if (!last_block(tickets + T_STEP)) return;
  double gc = 0.0, gb = 0.0, gx = 0.0;
  // one thread combines in block order: the partial count is small
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)gridDim.x; ++i) {
      gc += __ldcg(part + 3 * i);
      gb += __ldcg(part + 3 * i + 1);
      gx += __ldcg(part + 3 * i + 2);
    }
    sc->cx = gc;
    sc->by = gb;
    sc->xs = gx;
    sc->rel_gap = (gc - gb) / (1.0 + fabs(gc));
    tickets[T_STEP] = 0;
  }
}

__global__ void k_axpy(int64_t n, double a, const double* __restrict__ xv, double* yv, const Scalars* sc) {
  if (failed(sc)) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    yv[j] += a * xv[j];
}

// dot product into sc->dot_a (slot 0) or sc->dot_b (slot 1); fixed order.
__global__ void __launch_bounds__(kThreads) k_dot(int64_t n, const double* __restrict__ a,
                                                  const double* __restrict__ b, double* part, unsigned* tickets,
                                                  Scalars* sc, int slot) {
  __shared__ double sm[32];
  if (failed(sc)) return;
  double acc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    acc = fma(a[j], b[j], acc);
  acc = block_reduce<0>(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
  if (!last_block(tickets + T_DOT)) return;
  if (threadIdx.x == 0) {
    double g = 0.0;
    for (int i = 0; i < (int)gridDim.x; ++i) g += __ldcg(part + i);
    if (slot == 0) sc->dot_a = g; else sc->dot_b = g;
    tickets[T_DOT] = 0;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_diag_max(int64_t m, int64_t ldm, const T* __restrict__ M, double* part,
                                                       unsigned* tickets, Scalars* sc) {
  __shared__ double sm[32];
  double mx = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, fabs((double)M[p * ldm + p]));
  mx = block_reduce<1>(mx, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = mx;
  if (!last_block(tickets + T_NORM2)) return;
  double g = combine<1>(part, gridDim.x, sm);
  if (threadIdx.x == 0) {
    sc->mnorm = g;
    tickets[T_NORM2] = 0;
  }
}

__global__ void __launch_bounds__(kThreads) k_absmax(int64_t n, const double* __restrict__ v, double* part,
                                                     unsigned* tickets, Scalars* sc, int slot) {
  __shared__ double sm[32];
  if (failed(sc)) return;
  double mx = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double a = fabs(v[j]);
    mx = (a == a) ? fmax(mx, a) : INFINITY;
  }
  mx = block_reduce<1>(mx, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = mx;
  if (!last_block(tickets + T_NORM2)) return;
  double g = combine<1>(part, gridDim.x, sm);
  if (threadIdx.x == 0) {
    if (slot == 1) sc->rho_norm = g; else sc->dynorm = g;
    tickets[T_NORM2] = 0;
  }
}

template <typename T>
__global__ void k_gather_columns(int64_t m, int64_t n, const T* __restrict__ A, const double* __restrict__ D, int64_t k,
                                 const int* __restrict__ idx, T* __restrict__ Akept, double* __restrict__ Dkept) {
  const int64_t total = m * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / k, i = e % k;
    const int64_t j = idx[i];
    Akept[e] = A[p * n + j];
    if (p == 0) Dkept[i] = D[j];
  }
}

// out_p = sum_j A_pj^2 D_j = (A D A')_pp, one block per row (fixed order).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_normal_diag(int64_t m, int64_t n, const T* __restrict__ A,
                                                          const double* __restrict__ D, double* out,
                                                          const Scalars* sc) {
  __shared__ double sm[32];
  if (failed(sc)) return;
  for (int64_t p = blockIdx.x; p < m; p += gridDim.x) {
    const T* row = A + p * n;
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const double a = widen(row[j]);
      acc = fma(a * a, D[j], acc);
    }
    acc = block_reduce<0>(acc, sm);
    if (threadIdx.x == 0) out[p] = acc;
  }
}

__global__ void k_scale_vec(int64_t n, const double* __restrict__ D, const double* __restrict__ g, double* u,
                            const Scalars* sc) {
  if (failed(sc)) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    u[j] = D[j] * g[j];
}

__global__ void k_adjoint_lb(int64_t n, const double* __restrict__ D, const double* __restrict__ w,
                             const double* __restrict__ g, double* lb, const Scalars* sc) {
  if (failed(sc)) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    lb[j] = D[j] * (w[j] - g[j]);
}

__global__ void k_adjoint_init(int64_t n, const double* __restrict__ D, const double* __restrict__ w,
                               const double* __restrict__ g, const double* __restrict__ x, double* lb, double* lc,
                               double* wt, const Scalars* sc) {
  if (failed(sc)) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double b = D[j] * (w[j] - g[j]);
    lb[j] = b;
    lc[j] = -b / x[j];
    wt[j] = w[j];
  }
}

__global__ void k_adjoint_resid(int64_t n, const double* __restrict__ D, const double* __restrict__ g,
                                const double* __restrict__ x, const double* __restrict__ s,
                                const double* __restrict__ wt, const double* __restrict__ lb,
                                const double* __restrict__ lc, double* r1, double* r3, double* t, const Scalars* sc) {
  if (failed(sc)) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double a = g[j] - wt[j] - s[j] * lc[j];
    const double c = -lb[j] - x[j] * lc[j];
    r1[j] = a;
    r3[j] = c;
    t[j] = D[j] * a - c - lb[j];
  }
}

__global__ void k_adjoint_update(int64_t n, const double* __restrict__ D, const double* __restrict__ w,
                                 const double* __restrict__ x, const double* __restrict__ r1,
                                 const double* __restrict__ r3, double* lb, double* lc, double* wt,
                                 const Scalars* sc) {
  if (failed(sc)) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double db = D[j] * (w[j] - r1[j]) + r3[j];
    lb[j] += db;
    lc[j] += (r3[j] - db) / x[j];
    wt[j] += w[j];
  }
}

__global__ void k_adjoint_dA(int64_t m, int64_t n, const double* __restrict__ la, const double* __restrict__ x,
                             const double* __restrict__ y, const double* __restrict__ lb, double* dA,
                             const Scalars* sc) {
  if (failed(sc)) return;
  for (int64_t p = blockIdx.y; p < m; p += gridDim.y) {
    const double lp = la[p], yp = y[p];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
      dA[p * n + j] = -(lp * x[j] + yp * lb[j]);
  }
}

__global__ void k_krylov_update(int64_t n, const double* base, const double* __restrict__ p, double* out, int sign,
                                const Scalars* sc) {
  if (failed(sc)) return;
  const double coef = sc->dot_a / sc->dot_b;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = sign > 0 ? base[j] + coef * p[j] : base[j] - coef * p[j];
}

// p = z + (dot_a / beta_num) p
__global__ void k_krylov_direction(int64_t n, const double* __restrict__ z, double* p, double beta_den,
                                   const Scalars* sc) {
  if (failed(sc)) return;
  const double beta = sc->dot_a / beta_den;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    p[j] = z[j] + beta * p[j];
}

__global__ void k_convert_matrix(int64_t m, int64_t ld_src, const void* src, int src_f64, int64_t ld_dst, void* dst,
                                 int dst_f64) {
  for (int64_t i = blockIdx.y; i < m; i += gridDim.y)
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
      const double v = src_f64 ? ((const double*)src)[i * ld_src + j] : (double)((const float*)src)[i * ld_src + j];
      if (dst_f64) ((double*)dst)[i * ld_dst + j] = v;
      else ((float*)dst)[i * ld_dst + j] = (float)v;
    }
}


}  // namespace

// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_gemv(cudaStream_t st, int64_t m, int64_t n, const T* A, const double* v, const double* base,
                        double* out, double* part, unsigned* tickets, Scalars* sc, int norm_slot) {
  constexpr int ROWS = 4;
  const int64_t grid = (m + ROWS - 1) / ROWS;
  if (norm_slot >= 0 && grid > kPartMax) return cudaErrorInvalidConfiguration;
  k_gemv<T, ROWS><<<(unsigned)grid, kThreads, 0, st>>>(m, n, A, v, base, out, vec_aligned(A, n) ? 1 : 0, part,
                                                         tickets, sc, norm_slot);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gemv_t(cudaStream_t st, int64_t m, int64_t n, const T* A, const double* u, double* part,
                          int chunks, int64_t rows_per_chunk) {
  const bool vok = vec_aligned(A, n);
  const int64_t cols_per_block = (int64_t)kThreads * (vok ? Vec<T>::N : 1);
  dim3 grid((unsigned)((n + cols_per_block - 1) / cols_per_block), (unsigned)chunks);
  k_gemv_t_part<T><<<grid, kThreads, 0, st>>>(m, n, A, u, part, rows_per_chunk, vok ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_gemv_t_finish(cudaStream_t st, int64_t n, int chunks, const double* part, int mode,
                                 const double* x, const double* D, double* out0, double* out1, double* out2,
                                 const Scalars* sc, const double* rd) {
  k_gemv_t_finish<<<grid_for(n), kThreads, 0, st>>>(n, chunks, part, mode, x, D, out0, out1, out2, sc, rd);
  return cudaGetLastError();
}

cudaError_t launch_dual_residual(cudaStream_t st, int64_t n, const double* c, const double* s, const double* w,
                                 const double* D, double* rd, double* nu, const Scalars* sc) {
  k_dual_residual<<<grid_for(n), kThreads, 0, st>>>(n, c, s, w, D, rd, nu, sc);
  return cudaGetLastError();
}

cudaError_t launch_residual_norms(cudaStream_t st, int64_t m, int64_t n, const double* b, const double* rp,
                                  const double* c, const double* w, const double* s, double* part,
                                  unsigned* tickets, Scalars* sc) {
  k_residual_norms<<<grid_for(n > m ? n : m, 4), kThreads, 0, st>>>(m, n, b, rp, c, w, s, part, tickets, sc);
  return cudaGetLastError();
}

cudaError_t launch_scaling(cudaStream_t st, int64_t n, const double* x, const double* s, double* D, double* part,
                           unsigned* tickets, Scalars* sc) {
  const int g = grid_for(n, 4);
  k_scaling<<<g, kThreads, 0, st>>>(n, x, s, D, part, tickets, sc);
  return cudaGetLastError();
}

cudaError_t launch_psi(cudaStream_t st, int64_t n, const double* x, const double* s, const double* dx,
                       const double* ds, double alpha, double* part, unsigned* tickets, Scalars* sc,
                       bool capped) {
  k_psi<<<grid_for(n, 4), kThreads, 0, st>>>(n, x, s, dx, ds, alpha, part, tickets, sc, capped ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_step(cudaStream_t st, int64_t m, int64_t n, const double* b, const double* c, double* x,
                        double* y, double* s, const double* dx, const double* dy, const double* ds, double* part,
                        unsigned* tickets, Scalars* sc) {
  k_step<<<grid_for(n > m ? n : m, 4), kThreads, 0, st>>>(m, n, b, c, x, y, s, dx, dy, ds, part, tickets, sc);
  return cudaGetLastError();
}

cudaError_t launch_axpy(cudaStream_t st, int64_t n, double a, const double* xv, double* yv, const Scalars* sc) {
  k_axpy<<<grid_for(n), kThreads, 0, st>>>(n, a, xv, yv, sc);
  return cudaGetLastError();
}

cudaError_t launch_dot(cudaStream_t st, int64_t n, const double* a, const double* b, double* part,
                       unsigned* tickets, Scalars* sc, int slot) {
  k_dot<<<grid_for(n, 4), kThreads, 0, st>>>(n, a, b, part, tickets, sc, slot);
  return cudaGetLastError();
}

cudaError_t launch_krylov_update(cudaStream_t st, int64_t n, const double* base, const double* p, double* out,
                                 int sign, const Scalars* sc) {
  k_krylov_update<<<grid_for(n), kThreads, 0, st>>>(n, base, p, out, sign, sc);
  return cudaGetLastError();
}

cudaError_t launch_krylov_direction(cudaStream_t st, int64_t n, const double* z, double* p, double beta_den,
                                    const Scalars* sc) {
  k_krylov_direction<<<grid_for(n), kThreads, 0, st>>>(n, z, p, beta_den, sc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diag_max(cudaStream_t st, int64_t m, int64_t ldm, const T* M, double* part, unsigned* tickets,
                            Scalars* sc) {
  k_diag_max<T><<<grid_for(m, 4), kThreads, 0, st>>>(m, ldm, M, part, tickets, sc);
  return cudaGetLastError();
}
template cudaError_t launch_diag_max<double>(cudaStream_t, int64_t, int64_t, const double*, double*, unsigned*,
                                             Scalars*);
template cudaError_t launch_diag_max<float>(cudaStream_t, int64_t, int64_t, const float*, double*, unsigned*,
                                            Scalars*);

template <typename T>
cudaError_t launch_gather_columns(cudaStream_t st, int64_t m, int64_t n, const T* A, const double* D, int64_t k,
                                  const int* idx, T* Akept, double* Dkept) {
  k_gather_columns<T><<<grid_for(m * k, 4) * 4, kThreads, 0, st>>>(m, n, A, D, k, idx, Akept, Dkept);
  return cudaGetLastError();
}
template cudaError_t launch_gather_columns<double>(cudaStream_t, int64_t, int64_t, const double*, const double*,
                                                   int64_t, const int*, double*, double*);
template cudaError_t launch_gather_columns<float>(cudaStream_t, int64_t, int64_t, const float*, const double*, int64_t,
                                                  const int*, float*, double*);
template cudaError_t launch_gather_columns<__nv_bfloat16>(cudaStream_t, int64_t, int64_t, const __nv_bfloat16*,
                                                          const double*, int64_t, const int*, __nv_bfloat16*, double*);

cudaError_t launch_absmax(cudaStream_t st, int64_t n, const double* v, double* part, unsigned* tickets, Scalars* sc,
                          int slot) {
  k_absmax<<<grid_for(n, 4), kThreads, 0, st>>>(n, v, part, tickets, sc, slot);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_normal_diag(cudaStream_t st, int64_t m, int64_t n, const T* A, const double* D, double* out,
                               const Scalars* sc) {
  k_normal_diag<T><<<(unsigned)(m < 4 * 1184 ? m : 4 * 1184), kThreads, 0, st>>>(m, n, A, D, out, sc);
  return cudaGetLastError();
}
template cudaError_t launch_normal_diag<double>(cudaStream_t, int64_t, int64_t, const double*, const double*, double*,
                                                const Scalars*);
template cudaError_t launch_normal_diag<float>(cudaStream_t, int64_t, int64_t, const float*, const double*, double*,
                                               const Scalars*);
template cudaError_t launch_normal_diag<__nv_bfloat16>(cudaStream_t, int64_t, int64_t, const __nv_bfloat16*,
                                                       const double*, double*, const Scalars*);

cudaError_t launch_scale_vec(cudaStream_t st, int64_t n, const double* D, const double* g, double* u,
                             const Scalars* sc) {
  k_scale_vec<<<grid_for(n), kThreads, 0, st>>>(n, D, g, u, sc);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_lb(cudaStream_t st, int64_t n, const double* D, const double* w, const double* g,
                              double* lb, const Scalars* sc) {
  k_adjoint_lb<<<grid_for(n), kThreads, 0, st>>>(n, D, w, g, lb, sc);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_init(cudaStream_t st, int64_t n, const double* D, const double* w, const double* g,
                                const double* x, double* lb, double* lc, double* wt, const Scalars* sc) {
  k_adjoint_init<<<grid_for(n), kThreads, 0, st>>>(n, D, w, g, x, lb, lc, wt, sc);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_resid(cudaStream_t st, int64_t n, const double* D, const double* g, const double* x,
                                 const double* s, const double* wt, const double* lb, const double* lc, double* r1,
                                 double* r3, double* t, const Scalars* sc) {
  k_adjoint_resid<<<grid_for(n), kThreads, 0, st>>>(n, D, g, x, s, wt, lb, lc, r1, r3, t, sc);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_update(cudaStream_t st, int64_t n, const double* D, const double* w, const double* x,
                                  const double* r1, const double* r3, double* lb, double* lc, double* wt,
                                  const Scalars* sc) {
  k_adjoint_update<<<grid_for(n), kThreads, 0, st>>>(n, D, w, x, r1, r3, lb, lc, wt, sc);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_dA(cudaStream_t st, int64_t m, int64_t n, const double* la, const double* x,
                              const double* y, const double* lb, double* dA, const Scalars* sc) {
  dim3 grid((unsigned)((n + kThreads - 1) / kThreads < 64 ? (n + kThreads - 1) / kThreads : 64),
            (unsigned)(m < 4096 ? m : 4096));
  k_adjoint_dA<<<grid, kThreads, 0, st>>>(m, n, la, x, y, lb, dA, sc);
  return cudaGetLastError();
}

cudaError_t launch_convert_matrix(cudaStream_t st, int64_t m, int64_t ld_src, const void* src, int src_f64,
                                  int64_t ld_dst, void* dst, int dst_f64) {
  dim3 grid((unsigned)((m + kThreads - 1) / kThreads), (unsigned)(m < 4096 ? m : 4096));
  k_convert_matrix<<<grid, kThreads, 0, st>>>(m, ld_src, src, src_f64, ld_dst, dst, dst_f64);
  return cudaGetLastError();
}

#define PDAS_INST(T)                                                                                          \
  template cudaError_t launch_gemv<T>(cudaStream_t, int64_t, int64_t, const T*, const double*, const double*, \
                                      double*, double*, unsigned*, Scalars*, int);                            \
  template cudaError_t launch_gemv_t<T>(cudaStream_t, int64_t, int64_t, const T*, const double*, double*, int, \
                                        int64_t);
PDAS_INST(double)
PDAS_INST(float)
PDAS_INST(__nv_bfloat16)
#undef PDAS_INST

}  // namespace pdas
