/*
 * pdas_components.h -- step-by-step entry points of libpdas.
 *
 * Each call runs one stage of the Newton-direction solve of Eq. (3)/(4)
 * (N. Divakar, arXiv:1502.03543, Section V) on the handle's workspace, so a
 * caller or a test can check each stage on its own.  Conventions are those
 * of pdas.h: device pointers, the handle's stream, status codes, no traps.
 */
#ifndef PDAS_COMPONENTS_H
#define PDAS_COMPONENTS_H

#include "pdas.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Forms D = S^{-1} X (Eq. 4) and the lower triangle of the normal matrix
 * M = A D A' (Section V) in the workspace, in the handle's precision form
 * (FP64 for PDAS_FP64 or once a mixed form has switched to FP64; FP32 from
 * tensor-core or SIMT formation otherwise).  A: m x n (a_dtype); x, s: n. */
pdas_status pdas_form_normal(pdas_handle h, const void* A, const double* x, const double* s);

/* Copies the workspace matrix -- M after pdas_form_normal, the factor L
 * after pdas_factor -- to dst as a dense row-major m x m array (lower
 * triangle meaningful, the rest unspecified).  *dtype_out receives
 * PDAS_A_F64 (double) or PDAS_A_F32 (float), the element type written. */
pdas_status pdas_copy_matrix(pdas_handle h, void* dst, int* dtype_out);

/* Loads the lower triangle of src (row-major m x m, element type given by
 * dtype: PDAS_A_F64 or PDAS_A_F32, converted to the workspace precision)
 * into the workspace matrix. */
pdas_status pdas_load_matrix(pdas_handle h, const void* src, int dtype);

/* Blocked Cholesky M = L L' of the workspace matrix, in place (the
 * symmetric positive definite solve of Section V-A).  PDAS_ERR_NOT_SPD with
 * pdas_last_error_index = the first failing pivot if M is not SPD. */
pdas_status pdas_factor(pdas_handle h);

/* With the workspace factor: forward substitution L z = rhs, then back
 * substitution L' out = z.  rhs, out: m doubles (may alias). */
pdas_status pdas_factor_solve(pdas_handle h, const double* rhs, double* out);

/* Newton direction at (x, s) without stepping (Eq. 3 via Eq. 4):
 * dy solves (A D A') dy = A x (with FP64 refinement in mixed forms),
 * ds = -A' dy, dx = D(-ds) - x.  dx, ds: n; dy: m.  info may be NULL
 * (psi, theta, gap fields are not set). */
pdas_status pdas_direction(pdas_handle h, const void* A, const double* x, const double* s, double* dx, double* dy,
                           double* ds, pdas_iter_info* info);

/* The Newton direction of the infeasible-start variant at (x, y, s) (handle
 * created with opt.infeasible = 1, else PDAS_ERR_ARG): Eq. (3) with the
 * residuals r_p = b - A x and r_d = c - A'y - s as the right-hand sides of
 * its first two rows, reduced as in Section V: (A D A') dy = b + A D r_d,
 * ds = r_d - A' dy, dx = D(-ds) - x, with the handle's precision form and
 * refinement.  b (m), c (n), x, s (n), y (m): device doubles, unchanged.
 * dx, ds: n; dy: m.  info may be NULL (psi, theta, gap fields are not set). */
pdas_status pdas_direction_infeasible(pdas_handle h, const void* A, const double* b, const double* c,
                                      const double* x, const double* y, const double* s, double* dx, double* dy,
                                      double* ds, pdas_iter_info* info);

/* out (m) = A v (n), FP64 accumulation of exactly widened A: the right-hand
 * side A x of the normal equations.  On a mixed-form handle with A stored as
 * FP32 / BF16 (and exact_passes off) this is the double-float pass of the
 * refinement's operator (error within 2^-41 of sum |a v|). */
pdas_status pdas_gemv(pdas_handle h, const void* A, const double* v, double* out);

/* out (n) = A' u (m), FP64 accumulation: the product behind ds = -A' dy
 * (double-float on mixed-form handles, as pdas_gemv). */
pdas_status pdas_gemv_t(pdas_handle h, const void* A, const double* u, double* out);

/* Host-only, no GPU needed: the task order of the single-launch tile
 * Cholesky behind pdas_factor for FP32 factors (128 x 128 tiles, nb =
 * ceil(m / 128) tile rows), scheduled for nproc resident CTAs.  Writes
 * min(cap, count) tasks to out as int32 quadruples {kind, i, l, k}:
 * kind 0 = last update of diagonal tile (l, l) by tile column k = l - 1 (none
 * for l = 0), then its factorisation (i = l); 1 = last update of tile (i, l),
 * i >= l + 2, then its triangular solve against L_ll; 2 = update of tile
 * (i, l) by tile columns i and l of step k <= l - 2, or of step k = l - 1 when
 * i = l + 1; 3 = inverse of L_ll (for the blocked triangular solves); 4 =
 * triangular solve of the sub-diagonal tile (l + 1, l) against L_ll, all its
 * updates applied (k = l).  One CTA runs kinds 0 and 4 in the order 0(0),
 * 4(1,0), 0(1), 4(2,1), ...; the others take the rest in list order.  Returns
 * the count (0 for m <= 0); out may be NULL to query it.  Every task comes
 * after the tasks it waits for, which is what makes the launch
 * deadlock-free. */
int64_t pdas_chol_tile_tasks(int64_t m, int32_t nproc, int32_t* out, int64_t cap);

/* Size of the fixed device scratch behind pdas_gemv_t_noalloc: 8 MiB. */
#define PDAS_NOALLOC_SCRATCH_BYTES (8u << 20)

/* out (n) = A' u (m) like pdas_gemv_t, but with no handle and no device
 * allocation, for callers that cannot call cudaMalloc: code running while
 * another component captures the stream into a CUDA graph, processes whose
 * device memory belongs to another framework's pool, real-time loops that
 * forbid allocation after start-up.  The paper has no counterpart; this is a
 * deployment convenience.
 *   A: m x n row-major device array of dtype a_dtype (pdas_dtype); u: m
 *   doubles; out: n doubles (device, caller-owned); stream: cudaStream_t or
 *   NULL.  Results agree with pdas_gemv_t to FP64 summation-order rounding.
 * Scratch is one file-scope device array of PDAS_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until exit; n may be at most
 * (PDAS_NOALLOC_SCRATCH_BYTES - 256) / 8 = 1048544, else PDAS_ERR_ARG.  All
 * calls share that array, so calls that overlap on the GPU race: serialise
 * them.  The first call on a device fetches the array's device address
 * (with that device current) and loads the kernels; make it before any
 * stream capture.  That address is kept until the process exits, so it does
 * not survive cudaDeviceReset: do not call this entry point on a device
 * after resetting it.  Returns PDAS_OK, PDAS_ERR_ARG or PDAS_ERR_CUDA. */
pdas_status pdas_gemv_t_noalloc(int64_t m, int64_t n, int a_dtype, const void* A, const double* u, double* out,
                                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PDAS_COMPONENTS_H */
