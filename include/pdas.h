/*
 * pdas.h -- C ABI of libpdas, a GB300 (sm_103a) solver for the per-iteration
 * Newton direction of primal-dual affine scaling (PDAS).
 *
 * Method: N. Divakar, "Primal Dual Affine Scaling on GPUs", arXiv:1502.03543.
 *   Primal (Eq. 1): min c'x  s.t.  A x = b, x >= 0;   A is m x n, full rank,
 *   Dual   (Eq. 2): max b'y  s.t.  A'y + s = c, s >= 0;     m < n (Section I).
 *   Each iteration solves the Newton system Eq. (3) through its symmetric
 *   reduction Eq. (4), D = S^{-1} X, whose components are (Section V):
 *       (A D A') dy = A x,    ds = -A' dy,    dx = D(-ds) - x,
 *   then takes psi = max{ max_j(-dx_j/x_j), max_j(-ds_j/s_j) } and the step
 *   (x,y,s) += (alpha/psi)(dx,dy,ds), with alpha := 1 when psi <= 1
 *   ("Primal-Dual Affine Scaling" algorithm, Section III).
 *
 * Conventions for every entry point below:
 *   - Arrays are caller-owned DEVICE memory (e.g. PyTorch CUDA tensors),
 *     contiguous, 16-byte aligned.  A is dense row-major m x n in the dtype
 *     named by pdas_options.a_dtype; vectors are double.  The library never
 *     frees or retains caller pointers beyond the call.
 *   - The handle owns its workspace (normal matrix, factor, scratch), sized
 *     for (m, n) at pdas_create and released by pdas_destroy.  One handle
 *     serves one stream; do not share a handle between host threads.
 *   - All GPU work is ordered on pdas_options.stream.  pdas_step and
 *     pdas_solve synchronise that stream once per iteration to read the stop
 *     test (a few scalars); nothing else synchronises.
 *   - Errors come back as pdas_status codes; no entry point throws, traps or
 *     aborts.  A failing argument check modifies nothing.  After a
 *     PDAS_ERR_CUDA the handle should be destroyed.
 */
#ifndef PDAS_H
#define PDAS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdas_ctx* pdas_handle;

typedef enum {
  PDAS_OK = 0,
  PDAS_OPTIMAL = 1,         /* relative gap (c'x - b'y)/(1+|c'x|) below tol   */
  PDAS_OPTIMAL_EXACT = 2,   /* psi <= 1: full step taken onto the optimum      */
  PDAS_MAX_ITER = 3,        /* iteration cap reached                           */
  PDAS_STALLED = 4,         /* stall_count steps in a row shorter than stall_theta */
  PDAS_ZERO_DIRECTION = 5,  /* dx = dy = ds = 0 (the algorithm's literal stop) */
  PDAS_ERR_ARG = -1,        /* bad size, pointer, option or alpha              */
  PDAS_ERR_NOT_INTERIOR = -2, /* some x_j <= 0 or s_j <= 0                     */
  PDAS_ERR_NOT_SPD = -3,    /* Cholesky met a non-positive pivot (index: pdas_last_error_index) */
  PDAS_ERR_NONFINITE = -4,  /* NaN or Inf met in the iterate, direction or psi */
  PDAS_ERR_TIMEOUT = -5,    /* a bounded device-side wait gave up              */
  PDAS_ERR_CUDA = -6,       /* a CUDA runtime call failed (message: pdas_last_error_message) */
  PDAS_ERR_UNSUPPORTED = -7 /* entry point or option not available in this library */
} pdas_status;

/* Precision forms of the normal-equations solve. */
typedef enum {
  PDAS_FP64 = 0,    /* M = A D A' formed and factored in FP64                          */
  PDAS_TF32_IR = 1, /* M formed on tcgen05 tensor cores from TF32 operands (A and D.*A
                       split into TF32 parts each call, see splits; A stored as FP64 or
                       FP32), FP32 factor, FP64 refinement of dy                         */
  PDAS_BF16_IR = 2, /* as TF32_IR with BF16 operands (needs A stored as BF16)            */
  PDAS_FP32_IR = 3  /* M formed with FP32 SIMT arithmetic, FP32 factor, FP64 refinement  */
} pdas_form;

/* Storage dtype of A; every form reads A in this dtype and widens it exactly. */
typedef enum { PDAS_A_F64 = 0, PDAS_A_F32 = 1, PDAS_A_BF16 = 2 } pdas_dtype;

typedef struct {
  int form;                /* pdas_form                                             (PDAS_FP64) */
  int a_dtype;             /* pdas_dtype of A                                      (PDAS_A_F64) */
  int max_iter;            /* iteration cap of pdas_solve                                 (500) */
  double refine_tol;       /* refinement stops when ||Ax - M dy||_inf <= refine_tol ||Ax||_inf (1e-14) */
  int refine_max;          /* cap on refinement (preconditioned CG) steps per direction     (40) */
  double dspread_refactor; /* mixed forms: re-form and re-factor in FP64 for this and every later
                              iteration once max(D)/min(D) exceeds this (e.g. 1e8); <= 0 disables
                              the rule, leaving the switch to factor or refinement failure    (0) */
  void* stream;            /* cudaStream_t for all work; NULL = the legacy default stream      */
  int splits;              /* PDAS_BF16_IR: number of BF16 terms of D.*A (1..3), 0 = 3.
                              PDAS_TF32_IR: 0 or 3 = TF32 x 3 (A and D.*A split into hi + lo
                              TF32 parts, products hi hi + hi lo + lo hi: FP32-grade M); 1 = one
                              TF32 product (both rounded to TF32); 2: PDAS_ERR_UNSUPPORTED    */
  double stall_theta;      /* step length below which a step counts as stalled          (1e-12) */
  int stall_count;         /* consecutive stalled steps that end pdas_solve                  (5) */
  double refine_be;        /* refinement also stops when the normwise backward error
                              ||Ax - M dy||_inf / (max_p M_pp ||dy||_inf + ||Ax||_inf) <= refine_be;
                              0 disables                                                  (1e-14) */
  double drop_tol;         /* mixed forms in FP64: the factor is formed from the columns with
                              D_j >= drop_tol max(D) only (refinement still applies the whole
                              A D A'); 0 keeps every column                               (1e-10) */
  double drop_keep;        /* ... but never fewer than drop_keep * m columns (the largest D_j)  (1.25) */
  int exact_passes;        /* mixed forms with A stored as FP32 / BF16: 0 = the operator products
                              M p of the refinement's conjugate gradients while the factor is
                              FP32 (and pdas_gemv / pdas_gemv_t) run in double-float on the
                              FP32 pipes (FP32 pairs, FP64 accumulation every 16-32 terms),
                              several times faster on GB300; 1 = FP64.  The right-hand side,
                              the true residuals that decide acceptance and A' dy are FP64
                              either way                                                  (0) */
  int infeasible;          /* 0: the paper's system, which assumes a feasible interior start
                              (A x = b, A'y + s = c) and takes A x as the right-hand side of
                              the normal equations.  1: infeasible-start variant for any
                              interior (x, s) > 0: the rows A dx = 0 and A'dy + ds = 0 of
                              Eq. (3) take the residuals r_p = b - A x and r_d = c - A'y - s,
                              so (A D A') dy = b + A D r_d, ds = r_d - A'dy, dx = D(-ds) - x;
                              the step is theta = min(1, alpha/psi) (the iterate stays
                              interior; psi <= 1 ends nothing), and pdas_solve stops when
                              |rel_gap|, pres and dres (pdas_iter_info) are all below tol.
                              The variant has no centring term: from starts far from
                              feasibility it can stall at the boundary (PDAS_STALLED)   (0) */
  int fp64_tier_tc;        /* mixed forms in the FP64 tier: 1 = (a) with A stored as BF16, the
                              normal matrix of the kept columns (up to 16384 of them) is formed
                              on the tensor cores from exact fixed-point BF16 digit planes of A
                              and of D.*A (FP64-grade: products and sums exact, one FP64
                              rounding at the end; normal_form 4), and (b) for m > 256 the FP64
                              factor's trailing updates run on the tensor cores from digit
                              planes of each panel (FP64-grade at every gap);
                              0 = double-float formation (normal_form 2) and the factors of
                              df_factor_floor                                                 (1) */
  double df_factor_floor;  /* mixed forms in the FP64 tier without the tensor-core factor: the
                              factor is the double-float tile factor (FP32 pipes) while the
                              relative gap of the iterate is above this, the FP64 SIMT factor
                              below it; 0 = double-float to the end                        (1e-6) */
} pdas_options;

/* Per-iteration record of the last pdas_step (host memory, filled on return). */
typedef struct {
  double psi;           /* psi_k of the algorithm (Section III)                 */
  double theta;         /* step length used: alpha/psi, or 1 when psi <= 1 (infeasible-start
                           variant: min(1, alpha/psi))                          */
  double rel_gap;       /* (c'x - b'y)/(1+|c'x|) after the step                 */
  double cx, by, xs;    /* c'x, b'y, x's after the step                         */
  double dmax, dmin;    /* max and min of D = x/s before the step               */
  double refine_resid;  /* final ||Ax - M dy||_inf / ||Ax||_inf (mixed forms; 0 for FP64) */
  int refine_sweeps;    /* refinement sweeps taken (mixed forms)                */
  int used_fp64;        /* 1 if M was formed and factored in FP64 this iteration */
  int fp64_reason;      /* why a mixed form is in FP64: 0 not, 1 max(D)/min(D) rule,
                           2 low-precision factor not positive definite,
                           3 refinement did not reach its tolerance            */
  int64_t factor_columns; /* columns of A that formed the factor (n unless dropped) */
  int normal_form;      /* arithmetic of the normal matrix: 0 tcgen05 tensor cores, 1 FP32 SIMT,
                           2 double-float (FP32 pairs, ~48-bit) on the FP32 pipes, 3 FP64,
                           4 tcgen05 tensor cores on fixed-point digit planes (FP64-grade)       */
  double pres, dres;    /* infeasible-start variant: ||b - A x||_inf / (1 + ||b||_inf) and
                           ||c - A'y - s||_inf / (1 + ||c||_inf) after the step (else 0)        */
  int factor_form;      /* arithmetic of the factor of the accepted direction: 0 FP32 tile factor
                           (tensor-core products), 1 FP32 blocked SIMT, 2 double-float tile factor,
                           3 FP64 SIMT, 4 FP64 with tensor-core trailing updates from digit planes */
} pdas_iter_info;

/* Stages of one iteration, for pdas_profile. */
enum {
  PDAS_STAGE_RHS = 0,    /* D = x/s and r = A x                                    */
  PDAS_STAGE_NORMAL = 1, /* M = A D A' (lower triangle)                            */
  PDAS_STAGE_FACTOR = 2, /* Cholesky M = L L'                                      */
  PDAS_STAGE_SOLVE = 3,  /* triangular solves and FP64 refinement of dy           */
  PDAS_STAGE_DIR = 4,    /* ds = -A'dy, dx = D(-ds) - x                            */
  PDAS_STAGE_STEP = 5,   /* psi, theta and the step                                */
  PDAS_STAGE_FOLD = 6,   /* tensor-core forms: D.*A split into low-precision terms */
  PDAS_STAGE_COUNT = 7
};

/* Device time per stage, summed over the iterations since profiling was
 * enabled: CUDA events recorded on the handle's stream around each stage. */
typedef struct {
  double ms[PDAS_STAGE_COUNT];  /* summed milliseconds per stage              */
  int64_t calls[PDAS_STAGE_COUNT]; /* stage executions                        */
  int64_t launches;             /* kernels launched by the handle meanwhile    */
} pdas_profile;

/* Fills *opt with the defaults shown above. */
void pdas_default_options(pdas_options* opt);

/* Creates a handle for m x n problems (1 <= m < n, Section I) and allocates
 * its whole workspace on the current CUDA device, including the FP64 tier
 * of a mixed form (an FP64 m x m matrix and, with drop_tol > 0, an m x n
 * copy of the kept columns of A) and the adjoint's vectors: no later call
 * allocates device memory.  opt may be NULL (defaults).
 * Returns PDAS_ERR_ARG for bad sizes/options, PDAS_ERR_UNSUPPORTED for a
 * form/dtype pair that is not built, PDAS_ERR_CUDA if allocation fails. */
pdas_status pdas_create(int64_t m, int64_t n, const pdas_options* opt, pdas_handle* out);

/* One iteration of the algorithm of Section III: the Newton direction of
 * Eq. (3) via Eq. (4) at (x, s), the psi ratio test, and the step of length
 * theta = alpha/psi (theta = 1 when psi <= 1) applied in place to x (n),
 * y (m), s (n).  A: m x n device array; b (m), c (n): device doubles, used
 * for the gap.  0 < alpha < 1 (Section III).  info may be NULL.
 * Returns PDAS_OK to continue, PDAS_OPTIMAL_EXACT if psi <= 1, or an error;
 * on an error the iterate is left as it was before the call.  With
 * opt.infeasible the step is the variant's (see pdas_options): the residual
 * right-hand sides, theta = min(1, alpha/psi), never PDAS_OPTIMAL_EXACT, and
 * info->pres / dres hold the new iterate's relative residuals. */
pdas_status pdas_step(pdas_handle h, const void* A, const double* b, const double* c, double* x, double* y,
                      double* s, double alpha, pdas_iter_info* info);

/* Runs the algorithm of Section III from the interior point (x, y, s) until
 * the relative gap drops below tol (tested after each step; with
 * opt.infeasible, |gap| and both relative residuals below tol), psi <= 1, the
 * direction vanishes, stall, or max_iter.  x, y, s are updated in place to
 * the final iterate.  iters_out, rel_gap_out may be NULL.  Checks x > 0 and
 * s > 0 first (PDAS_ERR_NOT_INTERIOR, nothing modified). */
pdas_status pdas_solve(pdas_handle h, const void* A, const double* b, const double* c, double* x, double* y,
                       double* s, double alpha, double tol, int* iters_out, double* rel_gap_out);

/* Sensitivities of a loss L(x*) at a final iterate (x, y, s) of the
 * algorithm: implicit differentiation of F = [A x - b; A'y + s - c; X s - sigma]
 * = 0 with sigma = x.*s held fixed.  The adjoint of the Newton matrix of
 * Eq. (3) reduces, like the direction (Eq. 4), to the normal equations:
 *     (A D A') la = A D g,   lb = D (A' la - g),   D = X S^{-1},  g = dL/dx,
 * solved by FP64 conjugate gradients on A D A' (matrix-free) preconditioned
 * by the handle's last factor (so a pdas_step or pdas_solve must come first),
 * then refined on the full adjoint system with FP64 residuals (lb would
 * otherwise lose accuracy where D is large).
 * Outputs: dL_db (m) = la, dL_dc (n) = lb, dL_dA (m x n row-major, may be
 * NULL) = -(la x' + y lb').  A: m x n (a_dtype); x, y, s, dL_dx: device
 * doubles.  PDAS_ERR_ARG without a factor; PDAS_ERR_NOT_SPD if the
 * preconditioned solve breaks down. */
pdas_status pdas_backward(pdas_handle h, const void* A, const double* x, const double* y, const double* s,
                          const double* dL_dx, double* dL_dA, double* dL_db, double* dL_dc);

/* Releases the workspace and the handle.  NULL is ignored. */
void pdas_destroy(pdas_handle h);

/* Static English name of a status code. */
const char* pdas_status_str(pdas_status st);

/* Index that goes with the last error: the failing pivot for
 * PDAS_ERR_NOT_SPD, else -1. */
int64_t pdas_last_error_index(pdas_handle h);

/* Text of the last CUDA error seen by the handle ("" if none). */
const char* pdas_last_error_message(pdas_handle h);

/* Limit of every bounded inter-block wait of the handle's later calls, in
 * microseconds (failure detection; the paper has no counterpart): the
 * triangular solves' hand-offs between blocks and the tile Cholesky's
 * dependency waits give up after it, record PDAS_ERR_TIMEOUT and return,
 * leaving the handle usable.  0 restores the default of 2 s.  The waits on
 * the tensor-core pipelines' own barriers keep their fixed 2 s bound.
 * Synchronises the handle's stream.  PDAS_ERR_ARG if microseconds is
 * negative or above 2^31 - 1. */
pdas_status pdas_set_wait_limit(pdas_handle h, int64_t microseconds);

/* Starts (enable = 1) or stops (0) per-stage timing; starting clears the
 * accumulators and the launch count.  Timing adds one event record per
 * stage boundary and no synchronisation. */
pdas_status pdas_profile_enable(pdas_handle h, int enable);

/* Synchronises the handle's stream and returns the accumulated stage times
 * and the number of kernels the handle launched since profiling started. */
pdas_status pdas_profile_read(pdas_handle h, pdas_profile* out);

#ifdef __cplusplus
}
#endif

#endif /* PDAS_H */
