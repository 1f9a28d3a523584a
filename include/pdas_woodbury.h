/*
 * pdas_woodbury.h -- the paper's own solver of the normal equations, for
 * comparison with the Cholesky path of pdas.h.
 *
 * N. Divakar, "Primal Dual Affine Scaling on GPUs", arXiv:1502.03543,
 * Section V-A: only D changes between iterations, so A D A' is written as
 * the constant A A' plus the rank-one updates u_l v_l' with U = A and
 * V = A (D - I) (the Woodbury identity; the printed form of the identity is
 * garbled and is read as the standard one), and (A D A') x = r is solved by
 * the rank-one recurrence due to Egidi and Maponi:
 *     den_l   = 1 + v_l' y_{l-1,l},
 *     x_l     = x_{l-1}   - (v_l' x_{l-1}   / den_l) y_{l-1,l},
 *     y_{l,k} = y_{l-1,k} - (v_l' y_{l-1,k} / den_l) y_{l-1,l},  k = l+1..n,
 * from Y_0 = (A A')^{-1} A and x_0 = (A A')^{-1} r (the printed "x_0 = Y b"
 * is read as (A A')^{-1} applied to the right-hand side); x_n solves the
 * system.  O(m n^2) work per solve, against O(m^2 n) to form A D A'.  All
 * arithmetic is FP64.  The denominators den_l can come close to zero (an
 * intermediate matrix A A' + sum_{i<=l} u_i v_i' need not be definite, even
 * though A D A' is), and the recurrence then loses accuracy: the smallest
 * |den_l| is reported so the caller can judge.
 *
 * Conventions as in pdas.h: caller-owned device arrays (A m x n row-major
 * in the dtype given at create, vectors double), all work on the stream
 * given at create, status codes, no traps.  The handle owns A A' and its
 * factor (m x m), Y_0 and a working copy ((2n + 1) x m doubles), allocated
 * at create.  Limits: 1 <= m < n, m <= 14528 (two m-vectors of doubles per
 * block in shared memory).
 */
#ifndef PDAS_WOODBURY_H
#define PDAS_WOODBURY_H

#include <stdint.h>

#include "pdas.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdas_wb_ctx* pdas_wb_handle;

/* Creates a handle for m x n problems with A of dtype a_dtype (pdas_dtype);
 * stream: cudaStream_t or NULL.  PDAS_ERR_ARG for bad sizes, PDAS_ERR_CUDA
 * if allocation fails. */
pdas_status pdas_woodbury_create(int64_t m, int64_t n, int a_dtype, void* stream, pdas_wb_handle* out);

/* The part of Section V-A that does not depend on D, once per A: A A'
 * (FP64), its Cholesky factor, and Y_0 = (A A')^{-1} A (one forward and
 * back substitution per column).  PDAS_ERR_NOT_SPD if A A' is not positive
 * definite (A rank deficient). */
pdas_status pdas_woodbury_prepare(pdas_wb_handle h, const void* A);

/* x (m) = (A D A')^{-1} r (m) by the recurrence, D (n) the diagonal: n
 * launches, one per rank-one update.  A must be the matrix given to
 * pdas_woodbury_prepare (PDAS_ERR_ARG if prepare has not succeeded).
 * min_den_out (host, may be NULL) receives min_l |den_l|. */
pdas_status pdas_woodbury_solve(pdas_wb_handle h, const void* A, const double* D, const double* r, double* x,
                                double* min_den_out);

/* Text of the last CUDA error seen by the handle ("" if none). */
const char* pdas_woodbury_last_error_message(pdas_wb_handle h);

/* Releases the handle.  NULL is ignored. */
void pdas_woodbury_destroy(pdas_wb_handle h);

#ifdef __cplusplus
}
#endif

#endif /* PDAS_WOODBURY_H */
