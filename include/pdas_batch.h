/*
 * pdas_batch.h -- many small LPs solved by the PDAS algorithm of pdas.h
 * (N. Divakar, arXiv:1502.03543, Section III; Newton direction of Section V)
 * in one persistent launch per size bucket, replayed as one CUDA graph.
 *
 * Each LP i is min c_i'x s.t. A_i x = b_i, x >= 0 with 1 <= m_i < n_i,
 * m_i <= PDAS_BATCH_MAX_M and n_i <= PDAS_BATCH_MAX_N.  One CTA runs one LP
 * from its start to its stop, with the normal matrix M = A D A' (FP32) and
 * its Cholesky factor held in the CTA's shared memory; the direction is
 * refined to FP64 accuracy by preconditioned conjugate gradients on the
 * exact M.  Once the FP32 factor meets a non-positive pivot (near the
 * optimum, as max D / min D grows), the LP continues with M formed in
 * double-float and factored in FP64 in a global scratch slot.  CTAs take LPs from a
 * work queue, largest first.  LPs are grouped into buckets by m; every bucket
 * has its own launch (shared memory sized for the bucket) and its own CTA
 * size, chosen at creation by timing the candidates (pdas_batch_options.
 * autotune).  The launches of all buckets are captured once into a CUDA
 * graph (one branch per bucket) and replayed by every pdas_batch_solve.
 *
 * Buffers are caller-owned DEVICE memory bound to the handle for its whole
 * life (the graph holds their addresses): do not free them before
 * pdas_batch_destroy.  Packing, with offsets that are prefix sums in LP order:
 *   A    FP32, A_i row-major m_i x n_i at element offset sum_{k<i} m_k n_k;
 *   b, y double, m-vectors at offset sum_{k<i} m_k;
 *   c, x, s double, n-vectors at offset sum_{k<i} n_k.
 * (x, y, s) is the start on entry (strictly interior: x, s > 0) and the final
 * iterate on return, updated in place.
 */
#ifndef PDAS_BATCH_H
#define PDAS_BATCH_H

#include "pdas.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PDAS_BATCH_MAX_M 256
#define PDAS_BATCH_MAX_N 1024

typedef struct pdas_batch_ctx* pdas_batch_handle;

typedef struct {
  double alpha;       /* step fraction, 0 < alpha < 1                                 (0.95) */
  double tol;         /* stop when (c'x - b'y)/(1+|c'x|) < tol                        (1e-7) */
  int max_iter;       /* iteration cap per LP                                          (500) */
  double refine_tol;  /* refinement stops when ||Ax - M dy||_inf <= refine_tol ||Ax||_inf or
                         the normwise backward error is below it; every accepted residual
                         enters the iterate as primal drift (A dx = -(Ax - M dy))     (1e-14) */
  int refine_max;     /* conjugate-gradient steps per direction                         (40) */
  int autotune;       /* 1: time the candidate CTA sizes per bucket at creation (on
                         scratch copies of x, y, s); 0: use the built-in choice          (1) */
  void* stream;       /* cudaStream_t for all work; NULL = a stream the handle creates (the
                         solve graph cannot be captured on the legacy default stream)     */
} pdas_batch_options;

void pdas_batch_default_options(pdas_batch_options* opt);

/* Creates a handle for count LPs with sizes m[i], n[i] (host arrays) over the
 * bound device buffers described above; uploads the LP table, builds the
 * work queues, runs the autotuner if asked and captures the solve graph.
 * PDAS_ERR_ARG for bad sizes, pointers or options; PDAS_ERR_CUDA on a
 * runtime failure (message: pdas_batch_last_error_message). */
pdas_status pdas_batch_create(int count, const int* m, const int* n, const float* A, const double* b,
                              const double* c, double* x, double* y, double* s, const pdas_batch_options* opt,
                              pdas_batch_handle* out);

/* Runs every LP from its current iterate to its stop (replays the graph and
 * waits for it).  Per-LP results go to host arrays of count entries, each
 * may be NULL: status_out (pdas_status: OPTIMAL, OPTIMAL_EXACT, MAX_ITER,
 * STALLED, or an error such as ERR_NOT_INTERIOR / ERR_NOT_SPD /
 * ERR_NONFINITE for that LP alone), iters_out, gap_out (final relative gap).
 * Returns PDAS_OK when the launch completed, else the launch error. */
pdas_status pdas_batch_solve(pdas_batch_handle h, int* status_out, int* iters_out, double* gap_out);

/* Per-LP counters of the last pdas_batch_solve (host arrays of count
 * entries, each may be NULL): fp64_out = iterations run with the FP64 factor
 * (an LP moves to it for good once its FP32 factor meets a pivot that is not
 * positive); unrefined_out = iterations whose refinement stopped at
 * refine_max without meeting refine_tol (their direction is used as it
 * stands); time_us_out = device time of each LP's solve in microseconds
 * (its CTA's global timer, start to end). */
pdas_status pdas_batch_diagnostics(pdas_batch_handle h, int* fp64_out, int* unrefined_out, float* time_us_out);

/* The bucket layout: up to cap buckets, each with its upper bound on m, its
 * CTA size (threads) and its number of LPs.  Returns the bucket count. */
int pdas_batch_config(pdas_batch_handle h, int* m_bound, int* threads, int* lp_count, int cap);

/* Device time of the last pdas_batch_solve in milliseconds (CUDA events on
 * the handle's stream around the graph), or a negative value. */
double pdas_batch_last_ms(pdas_batch_handle h);

const char* pdas_batch_last_error_message(pdas_batch_handle h);

/* Sensitivities of a loss L(x*_1, ..., x*_count) at every LP's final
 * iterate, after pdas_batch_solve, in one launch per bucket (one CTA per LP,
 * as the solve): the adjoint of pdas_backward (pdas.h) for each LP --
 * implicit differentiation of F = [A x - b; A'y + s - c; X s - sigma] = 0
 * with sigma = x.*s held fixed, reduced to the normal equations of the
 * Newton direction (Section V), (A D A') la = A D g, lb = D (A' la - g),
 * and refined twice on the full adjoint system with FP64 residuals.  The
 * normal matrix at the final D is formed and factored in the CTA (FP32, or
 * the FP64 tier's factor where the FP32 one fails) to precondition the
 * solves.  Device arrays, packed like the handle's buffers: dL_dx (like x,
 * g = dL/dx), dL_db (like b) = la, dL_dc (like c) = lb, and dL_dA (FP64,
 * packed like A; may be NULL) = -(la x' + y lb').  status_out (host, count
 * entries, may be NULL) receives each LP's status: PDAS_OK, or
 * PDAS_ERR_NOT_SPD if its solve broke down, PDAS_ERR_NOT_INTERIOR.  Returns
 * PDAS_OK when the launches completed. */
pdas_status pdas_batch_backward(pdas_batch_handle h, const double* dL_dx, double* dL_dA, double* dL_db,
                                double* dL_dc, int* status_out);

void pdas_batch_destroy(pdas_batch_handle h);

#ifdef __cplusplus
}
#endif

#endif /* PDAS_BATCH_H */
