/*
 * pdas_oracle.c -- plain FP64 CPU oracle for primal-dual affine scaling (PDAS).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, constant or helper with the CUDA path, and it never calls it.
 *
 * Source: N. Divakar, "Primal Dual Affine Scaling on GPUs" (arXiv:1502.03543).
 *   - Problem: primal Eq. (1) min c'x s.t. Ax=b, x>=0; dual Eq. (2)
 *     max b'y s.t. A'y+s=c, s>=0; A is m x n, full rank, m<n (Section I).
 *   - Newton system Eq. (3) and its symmetric reduction Eq. (4) with
 *     D = S^{-1} X, whose components are (Section V):
 *         dx = D(-ds) - x,   (A D A') dy = A x,   ds = -A' dy.
 *   - Outer loop: the "Primal-Dual Affine Scaling" algorithm of Section III
 *     (psi ratio test, step alpha/psi, stop on psi = 1).
 *
 * Readings where the paper is silent or garbled (each one also listed in the
 * design notes):
 *   R1  X_k^{-}1 in the psi line of the algorithm is X_k^{-1}.
 *   R2  The stop "dx=dy=ds=0" cannot be reached from an interior point; it is
 *       kept literally and the relative-gap test
 *       (c'x - b'y) / (1 + |c'x|) < tol is added, tested after each step.
 *   R3  The right-hand side of the normal equations is A x, as printed
 *       (not b).
 *   R4  "psi = 1" is read as psi <= 1: then theta = 1 (alpha := 1) and the
 *       solver stops after the step.  Otherwise theta = alpha / psi.
 *   R10 The paper gives no iteration cap; max_iter is an argument, and the
 *       run is declared stalled after 5 consecutive steps with theta < 1e-12.
 *   R11 Infeasible-start variant (not in the paper, which assumes a feasible
 *       interior start): the rows A dx = 0 and A' dy + ds = 0 of Eq. (3)
 *       take the residuals r_p = b - A x and r_d = c - A' y - s as their
 *       right-hand sides.  The reduction of Section V then gives
 *       (A D A') dy = b + A D r_d, ds = r_d - A' dy, dx = D(-ds) - x; from a
 *       feasible start it is the paper's system.  A full step from an
 *       infeasible point does not end at an optimum, so the variant steps
 *       theta = min(1, alpha / psi) (the iterate stays interior), never stops
 *       on psi, and stops when |rel_gap|, ||r_p||_inf / (1 + ||b||_inf) and
 *       ||r_d||_inf / (1 + ||c||_inf) are all below tol.
 *
 * Arithmetic: every sum runs left to right in increasing index order, in
 * FP64, with no fused multiply-add (build with -ffp-contract=off).  OpenMP is
 * used only across independent outputs (rows of M, entries of A v, columns
 * of L below a pivot), never inside one sum, so the result does not depend
 * on the thread count.  Dense A is row-major m x n; M and L are row-major
 * m x m.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OPTIMAL 1       /* relative gap below tol (reading R2)          */
#define OR_OPTIMAL_EXACT 2 /* psi <= 1: full step taken (reading R4)        */
#define OR_MAX_ITER 3
#define OR_STALLED 4
#define OR_ZERO_DIRECTION 5 /* the paper's literal stop dx=dy=ds=0         */
#define OR_NOT_SPD -3

int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* D = S^{-1} X (Eq. (4)): D_j = x_j / s_j. */
void or_scaling(int64_t n, const double* x, const double* s, double* D) {
  for (int64_t j = 0; j < n; ++j) D[j] = x[j] / s[j];
}

/* out = A v: the right-hand side A x of the normal equations (Section V). */
void or_gemv(int64_t m, int64_t n, const double* A, const double* v, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < m; ++p) {
    const double* a = A + p * n;
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j) acc += a[j] * v[j];
    out[p] = acc;
  }
}

/* out = A' v, as in ds = -A' dy (Section V). */
void or_gemv_t(int64_t m, int64_t n, const double* A, const double* v, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    double acc = 0.0;
    for (int64_t p = 0; p < m; ++p) acc += A[p * n + j] * v[p];
    out[j] = acc;
  }
}

/* One entry of the normal matrix M = A D A' (Section V):
 * M_pq = sum_j A_pj D_j A_qj, summed in increasing j. */
double or_normal_entry(int64_t m, int64_t n, const double* A, const double* D, int64_t p, int64_t q) {
  (void)m;
  const double* ap = A + p * n;
  const double* aq = A + q * n;
  double acc = 0.0;
  for (int64_t j = 0; j < n; ++j) acc += (ap[j] * D[j]) * aq[j];
  return acc;
}

/* Rows [p0, p1) of the normal matrix, lower triangle q <= p, written into the
 * row-major m x m array M (entries above the diagonal are left untouched). */
void or_normal_rows(int64_t m, int64_t n, const double* A, const double* D, int64_t p0, int64_t p1,
                    double* M) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = p0; p < p1; ++p)
    for (int64_t q = 0; q <= p; ++q) M[p * m + q] = or_normal_entry(m, n, A, D, p, q);
}

/* Full symmetric M = A D A' (both triangles). */
void or_normal_matrix(int64_t m, int64_t n, const double* A, const double* D, double* M) {
  or_normal_rows(m, n, A, D, 0, m, M);
  for (int64_t p = 0; p < m; ++p)
    for (int64_t q = p + 1; q < m; ++q) M[p * m + q] = M[q * m + p];
}

/* Cholesky M = L L' of the symmetric positive definite normal matrix
 * (Section V-A names Cholesky as the usual way to solve (A D A') dy = A x).
 * Column by column: L_jj = sqrt(M_jj - sum_{k<j} L_jk^2),
 * L_ij = (M_ij - sum_{k<j} L_ik L_jk) / L_jj for i > j.  Reads the lower
 * triangle of M only; writes the full L (zeros above the diagonal).
 * Returns -1 on success, else the index j of the first pivot that is not
 * positive (or not finite); L is then only partially written. */
int64_t or_cholesky(int64_t m, const double* M, double* L) {
  memset(L, 0, (size_t)(m * m) * sizeof(double));
  for (int64_t j = 0; j < m; ++j) {
    const double* lj = L + j * m;
    double d = M[j * m + j];
    for (int64_t k = 0; k < j; ++k) d -= lj[k] * lj[k];
    if (!(d > 0.0) || !isfinite(d)) return j;
    const double ljj = sqrt(d);
    L[j * m + j] = ljj;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < m; ++i) {
      const double* li = L + i * m;
      double acc = M[i * m + j];
      for (int64_t k = 0; k < j; ++k) acc -= li[k] * lj[k];
      L[i * m + j] = acc / ljj;
    }
  }
  return -1;
}

/* Forward substitution L z = v. */
void or_forward(int64_t m, const double* L, const double* v, double* z) {
  for (int64_t i = 0; i < m; ++i) {
    const double* li = L + i * m;
    double acc = v[i];
    for (int64_t k = 0; k < i; ++k) acc -= li[k] * z[k];
    z[i] = acc / li[i];
  }
}

/* Back substitution L' y = z. */
void or_backward(int64_t m, const double* L, const double* z, double* y) {
  for (int64_t i = m - 1; i >= 0; --i) {
    double acc = z[i];
    for (int64_t k = i + 1; k < m; ++k) acc -= L[k * m + i] * y[k];
    y[i] = acc / L[i * m + i];
  }
}

/* Newton direction of Eq. (3) through its symmetric reduction Eq. (4):
 *   D = x/s, r = A x, M = A D A', M dy = r (Cholesky), w = A' dy,
 *   ds = -w, dx = D(-ds) - x.
 * D_out, r_out, M_out, L_out may be NULL.  Returns -1, or the failing pivot. */
int64_t or_direction(int64_t m, int64_t n, const double* A, const double* x, const double* s, double* dx,
                     double* dy, double* ds, double* D_out, double* r_out, double* M_out, double* L_out) {
  double* D = (double*)malloc((size_t)n * sizeof(double));
  double* r = (double*)malloc((size_t)m * sizeof(double));
  double* w = (double*)malloc((size_t)n * sizeof(double));
  double* z = (double*)malloc((size_t)m * sizeof(double));
  double* M = M_out ? M_out : (double*)malloc((size_t)(m * m) * sizeof(double));
  double* L = L_out ? L_out : (double*)malloc((size_t)(m * m) * sizeof(double));
  or_scaling(n, x, s, D);
  or_gemv(m, n, A, x, r);
  or_normal_matrix(m, n, A, D, M);
  int64_t fail = or_cholesky(m, M, L);
  if (fail < 0) {
    or_forward(m, L, r, z);
    or_backward(m, L, z, dy);
    or_gemv_t(m, n, A, dy, w);
    for (int64_t j = 0; j < n; ++j) {
      ds[j] = -w[j];
      dx[j] = D[j] * (-ds[j]) - x[j];
    }
  }
  if (D_out) memcpy(D_out, D, (size_t)n * sizeof(double));
  if (r_out) memcpy(r_out, r, (size_t)m * sizeof(double));
  if (!M_out) free(M);
  if (!L_out) free(L);
  free(D); free(r); free(w); free(z);
  return fail;
}

/* Newton direction of the infeasible-start variant (reading R11):
 *   D = x/s, r_d = c - A' y - s, r = b + A (D r_d), M = A D A', M dy = r,
 *   w = A' dy, ds = r_d - w, dx = D(-ds) - x.
 * D_out, r_out, rd_out may be NULL.  Returns -1, or the failing pivot. */
int64_t or_direction_infeasible(int64_t m, int64_t n, const double* A, const double* b, const double* c,
                                const double* x, const double* y, const double* s, double* dx, double* dy,
                                double* ds, double* D_out, double* r_out, double* rd_out) {
  double* D = (double*)malloc((size_t)n * sizeof(double));
  double* rd = (double*)malloc((size_t)n * sizeof(double));
  double* u = (double*)malloc((size_t)n * sizeof(double));
  double* w = (double*)malloc((size_t)n * sizeof(double));
  double* r = (double*)malloc((size_t)m * sizeof(double));
  double* z = (double*)malloc((size_t)m * sizeof(double));
  double* M = (double*)malloc((size_t)(m * m) * sizeof(double));
  double* L = (double*)malloc((size_t)(m * m) * sizeof(double));
  or_scaling(n, x, s, D);
  or_gemv_t(m, n, A, y, w);
  for (int64_t j = 0; j < n; ++j) {
    rd[j] = (c[j] - w[j]) - s[j];
    u[j] = D[j] * rd[j];
  }
  or_gemv(m, n, A, u, z);
  for (int64_t p = 0; p < m; ++p) r[p] = b[p] + z[p];
  or_normal_matrix(m, n, A, D, M);
  int64_t fail = or_cholesky(m, M, L);
  if (fail < 0) {
    or_forward(m, L, r, z);
    or_backward(m, L, z, dy);
    or_gemv_t(m, n, A, dy, w);
    for (int64_t j = 0; j < n; ++j) {
      ds[j] = rd[j] - w[j];
      dx[j] = -D[j] * ds[j] - x[j]; /* = D(-ds) - x exactly */
    }
  }
  if (D_out) memcpy(D_out, D, (size_t)n * sizeof(double));
  if (r_out) memcpy(r_out, r, (size_t)m * sizeof(double));
  if (rd_out) memcpy(rd_out, rd, (size_t)n * sizeof(double));
  free(D); free(rd); free(u); free(w); free(r); free(z); free(M); free(L);
  return fail;
}

/* Relative residuals of (x, y, s) (reading R11):
 * out[0] = ||b - A x||_inf / (1 + ||b||_inf), out[1] = ||c - A' y - s||_inf / (1 + ||c||_inf). */
void or_residuals(int64_t m, int64_t n, const double* A, const double* b, const double* c, const double* x,
                  const double* y, const double* s, double* out) {
  double* t = (double*)malloc((size_t)m * sizeof(double));
  double* w = (double*)malloc((size_t)n * sizeof(double));
  or_gemv(m, n, A, x, t);
  or_gemv_t(m, n, A, y, w);
  double rp = 0.0, bn = 0.0, rdn = 0.0, cn = 0.0;
  for (int64_t p = 0; p < m; ++p) {
    rp = fmax(rp, fabs(b[p] - t[p]));
    bn = fmax(bn, fabs(b[p]));
  }
  for (int64_t j = 0; j < n; ++j) {
    rdn = fmax(rdn, fabs((c[j] - w[j]) - s[j]));
    cn = fmax(cn, fabs(c[j]));
  }
  out[0] = rp / (1.0 + bn);
  out[1] = rdn / (1.0 + cn);
  free(t); free(w);
}

/* psi = max{ phi(-X^{-1} dx), phi(-S^{-1} ds) }, phi(u) = max_j u_j
 * (Section III, reading R1). */
double or_psi(int64_t n, const double* x, const double* s, const double* dx, const double* ds) {
  double psi = -INFINITY;
  for (int64_t j = 0; j < n; ++j) {
    double u = -dx[j] / x[j];
    double v = -ds[j] / s[j];
    if (u > psi) psi = u;
    if (v > psi) psi = v;
  }
  return psi;
}

/* Step length of the algorithm: alpha/psi, or 1 when psi <= 1 (reading R4). */
double or_theta(double psi, double alpha) { return psi <= 1.0 ? 1.0 : alpha / psi; }

/* Step length of the infeasible-start variant (reading R11): min(1, alpha/psi). */
double or_theta_infeasible(double psi, double alpha) { return psi <= alpha ? 1.0 : alpha / psi; }

/* (x,y,s) += theta (dx,dy,ds). */
void or_step(int64_t m, int64_t n, double theta, double* x, double* y, double* s, const double* dx,
             const double* dy, const double* ds) {
  for (int64_t j = 0; j < n; ++j) x[j] = x[j] + theta * dx[j];
  for (int64_t p = 0; p < m; ++p) y[p] = y[p] + theta * dy[p];
  for (int64_t j = 0; j < n; ++j) s[j] = s[j] + theta * ds[j];
}

static double dot(int64_t n, const double* a, const double* b) {
  double acc = 0.0;
  for (int64_t j = 0; j < n; ++j) acc += a[j] * b[j];
  return acc;
}

/* Relative duality gap (reading R2): (c'x - b'y) / (1 + |c'x|). */
double or_rel_gap(int64_t m, int64_t n, const double* b, const double* c, const double* x, const double* y) {
  double cx = dot(n, c, x);
  double by = dot(m, b, y);
  return (cx - by) / (1.0 + fabs(cx));
}

/* The "Primal-Dual Affine Scaling" algorithm of Section III.
 *
 * x (n), y (m), s (n) hold the interior start on entry and the final iterate
 * on return.  trace, if not NULL, receives per iteration k the 4 values
 * {psi_k, theta_k, rel_gap after the step, max D / min D}; iterates, if not
 * NULL, receives per iteration the iterate after the step as
 * [x (n) | y (m) | s (n)].  Both must hold max_iter records.
 * *iters_out = number of Newton directions computed.
 * *fail_index_out = failing pivot index on OR_NOT_SPD, else -1.
 * infeasible != 0 runs the infeasible-start variant (reading R11); then
 * res_trace, if not NULL, receives per iteration the 2 relative residuals
 * of or_residuals after the step.
 * Returns one of the OR_* codes above. */
int or_solve(int64_t m, int64_t n, const double* A, const double* b, const double* c, double* x, double* y,
             double* s, double alpha, double tol, int max_iter, int* iters_out, double* trace,
             double* iterates, int64_t* fail_index_out, int infeasible, double* res_trace) {
  double* dx = (double*)malloc((size_t)n * sizeof(double));
  double* dy = (double*)malloc((size_t)m * sizeof(double));
  double* ds = (double*)malloc((size_t)n * sizeof(double));
  double* D = (double*)malloc((size_t)n * sizeof(double));
  int status = OR_MAX_ITER, small_steps = 0, k;
  *fail_index_out = -1;
  for (k = 0; k < max_iter; ++k) {
    int64_t fail = infeasible ? or_direction_infeasible(m, n, A, b, c, x, y, s, dx, dy, ds, D, NULL, NULL)
                              : or_direction(m, n, A, x, s, dx, dy, ds, D, NULL, NULL, NULL);
    if (fail >= 0) {
      *fail_index_out = fail;
      status = OR_NOT_SPD;
      break;
    }
    /* The paper's literal stop: all three directions zero. */
    int zero = 1;
    for (int64_t j = 0; j < n && zero; ++j) zero = (dx[j] == 0.0 && ds[j] == 0.0);
    for (int64_t p = 0; p < m && zero; ++p) zero = (dy[p] == 0.0);
    if (zero) {
      status = OR_ZERO_DIRECTION;
      ++k;
      break;
    }
    double psi = or_psi(n, x, s, dx, ds);
    double theta = infeasible ? or_theta_infeasible(psi, alpha) : or_theta(psi, alpha);
    or_step(m, n, theta, x, y, s, dx, dy, ds);
    double gap = or_rel_gap(m, n, b, c, x, y);
    double res[2] = {0.0, 0.0};
    if (infeasible) {
      or_residuals(m, n, A, b, c, x, y, s, res);
      if (res_trace) {
        res_trace[2 * k + 0] = res[0];
        res_trace[2 * k + 1] = res[1];
      }
    }
    if (trace) {
      double dmax = D[0], dmin = D[0];
      for (int64_t j = 1; j < n; ++j) {
        if (D[j] > dmax) dmax = D[j];
        if (D[j] < dmin) dmin = D[j];
      }
      trace[4 * k + 0] = psi;
      trace[4 * k + 1] = theta;
      trace[4 * k + 2] = gap;
      trace[4 * k + 3] = dmax / dmin;
    }
    if (iterates) {
      double* it = iterates + (size_t)k * (size_t)(2 * n + m);
      memcpy(it, x, (size_t)n * sizeof(double));
      memcpy(it + n, y, (size_t)m * sizeof(double));
      memcpy(it + n + m, s, (size_t)n * sizeof(double));
    }
    if (infeasible) {
      if (fabs(gap) < tol && res[0] < tol && res[1] < tol) {
        status = OR_OPTIMAL;
        ++k;
        break;
      }
    } else if (psi <= 1.0) {
      status = OR_OPTIMAL_EXACT;
      ++k;
      break;
    } else if (gap < tol) {
      status = OR_OPTIMAL;
      ++k;
      break;
    }
    small_steps = theta < 1e-12 ? small_steps + 1 : 0;
    if (small_steps >= 5) {
      status = OR_STALLED;
      ++k;
      break;
    }
  }
  *iters_out = k;
  free(dx); free(dy); free(ds); free(D);
  return status;
}
