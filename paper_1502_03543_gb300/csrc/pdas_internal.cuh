// pdas_internal.cuh -- shared declarations of the libpdas CUDA sources.
//
// Layout in HBM (all row-major, all resident for the life of a handle):
//   A       m x n, caller-owned, in its storage dtype (f64 / f32 / bf16);
//   M, L    m x m with leading dimension ldm = round_up(m, 16), lower
//           triangle only; L overwrites M in place;
//   vectors D, r, dy, w, ... in FP64.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pdas.h"
#include "pdas_components.h"

namespace pdas {

constexpr int kThreads = 256;   // threads of every elementwise / reduction kernel
constexpr int kTile = 64;       // SIMT SYRK / Cholesky tile edge
constexpr int kPartMax = 65536;  // capacity of the reduction-partials buffer (blocks)

// Scalars written by the device reductions; the host reads the whole struct
// once per iteration.
struct Scalars {
  double dmax, dmin;   // max, min of D = x/s
  double psi, theta;   // ratio test and step length
  double cx, by, xs;   // c'x, b'y, x's after the step
  double rel_gap;      // (c'x - b'y)/(1+|c'x|)
  double rnorm;        // ||A x||_inf
  double rho_norm;     // ||A x - M dy||_inf of the latest residual
  double dot_a, dot_b; // dot products of the refinement Krylov steps
  double mnorm;        // max_p M_pp of the formed normal matrix (a lower bound on ||M||)
  double dynorm;       // ||dy||_inf
  double pres, dres;   // infeasible-start variant: relative primal and dual residuals
  int status;          // 0, or a pdas_status error detected on the device
  int fail_index;      // failing pivot for PDAS_ERR_NOT_SPD
  int bad_iterate;     // nonzero if some x_j <= 0 or s_j <= 0 (or not finite)
  int wait_us;         // limit of the bounded inter-block waits in microseconds (0: 2 s)
};

// Counters for the "last block finishes the reduction" pattern and the
// triangular-solve tickets.
enum Ticket { T_SCALING = 0, T_PSI, T_STEP, T_NORM, T_NORM2, T_DOT, T_TRSV, T_CHOL, T_RES, T_COUNT = 9 };

// ---- exact widening of the stored A ---------------------------------------
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return (double)v; }
__device__ __forceinline__ double widen(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
// FP32 -> FP64 widening by bit manipulation on the integer pipes: on GB300
// the FP64 pipe is the bound of every pass over A, and a conversion
// instruction would occupy it as long as the multiply-add does.  Exact for
// every FP32 value: normal numbers move their exponent from bias 127 to
// 1023, zeros keep their sign, Inf/NaN map to exponent 2047; subnormals take
// the conversion instruction (they do not occur in practice).
__device__ __forceinline__ double widen_bits(uint32_t u) {
  const uint32_t e = (u >> 23) & 0xffu;
  const uint32_t mant = u & 0x7fffffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0u) {
    if (mant == 0u) return __longlong_as_double((long long)sign);
    return (double)__uint_as_float(u);
  }
  const unsigned long long e64 = (e == 0xffu) ? 2047ull : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(sign | (e64 << 52) | ((unsigned long long)mant << 29)));
}

__device__ __forceinline__ float widen32(double v) { return (float)v; }
__device__ __forceinline__ float widen32(float v) { return v; }
__device__ __forceinline__ float widen32(__nv_bfloat16 v) { return __bfloat162float(v); }

// ---- launch helpers (host) ------------------------------------------------
// Each returns cudaGetLastError() of its launch.
template <typename T>
cudaError_t launch_gemv(cudaStream_t st, int64_t m, int64_t n, const T* A, const double* v, const double* base,
                        double* out, double* part, unsigned* tickets, Scalars* sc, int norm_slot);
template <typename T>
cudaError_t launch_gemv_t(cudaStream_t st, int64_t m, int64_t n, const T* A, const double* u, double* part,
                          int chunks, int64_t rows_per_chunk);

// The passes over A in double-float on the FP32 pipes (gemv_df.cu), for A
// stored as FP32 or BF16: v (or u) is first split into FP32 pairs by
// launch_split_pairs; results and partials are FP64 as above.
cudaError_t launch_split_pairs(cudaStream_t st, int64_t n, const double* v, float2* out);
template <typename T>
cudaError_t launch_gemv_df(cudaStream_t st, int64_t m, int64_t n, const T* A, const float2* v2, const double* base,
                           double* out, double* part, unsigned* tickets, Scalars* sc, int norm_slot);
template <typename T>
cudaError_t launch_gemv_t_df(cudaStream_t st, int64_t m, int64_t n, const T* A, const float2* u2, double* part,
                             int chunks, int64_t rows_per_chunk);
// w = sum of the gemv_t partials; then per mode:
//   0: out0 = w
//   1: direction: out0 = dx = D w - x, out1 = ds = -w, out2 = w (may be null)
//   2: scaled:    out0 = D w, out2 = w (may be null)
//   3: direction from a w already in out2 (chunks, part unused)
// With rd (modes 1 and 3, the infeasible-start variant) ds = rd - w instead of -w.
cudaError_t launch_gemv_t_finish(cudaStream_t st, int64_t n, int chunks, const double* part, int mode,
                                 const double* x, const double* D, double* out0, double* out1, double* out2,
                                 const Scalars* sc, const double* rd = nullptr);
// Infeasible-start variant: rd = (c - w) - s (w = A'y) and nu = -(D rd), so
// that b - A nu = b + A D rd is the right-hand side of the normal equations.
cudaError_t launch_dual_residual(cudaStream_t st, int64_t n, const double* c, const double* s, const double* w,
                                 const double* D, double* rd, double* nu, const Scalars* sc);
// sc->pres = max|rp| / (1 + max|b|) with rp = b - A x (m), sc->dres =
// max|(c - w) - s| / (1 + max|c|) with w = A'y (n).
cudaError_t launch_residual_norms(cudaStream_t st, int64_t m, int64_t n, const double* b, const double* rp,
                                  const double* c, const double* w, const double* s, double* part,
                                  unsigned* tickets, Scalars* sc);
cudaError_t launch_scaling(cudaStream_t st, int64_t n, const double* x, const double* s, double* D, double* part,
                           unsigned* tickets, Scalars* sc);
// capped: theta = min(1, alpha/psi) (infeasible-start variant) instead of 1 when psi <= 1.
cudaError_t launch_psi(cudaStream_t st, int64_t n, const double* x, const double* s, const double* dx,
                       const double* ds, double alpha, double* part, unsigned* tickets, Scalars* sc,
                       bool capped = false);
cudaError_t launch_step(cudaStream_t st, int64_t m, int64_t n, const double* b, const double* c, double* x,
                        double* y, double* s, const double* dx, const double* dy, const double* ds, double* part,
                        unsigned* tickets, Scalars* sc);
cudaError_t launch_axpy(cudaStream_t st, int64_t n, double a, const double* xv, double* yv, const Scalars* sc);
cudaError_t launch_dot(cudaStream_t st, int64_t n, const double* a, const double* b, double* part,
                       unsigned* tickets, Scalars* sc, int slot);
// x-update of one Krylov step: out = base + coef * p where coef = sc->dot_a / sc->dot_b
// (sign < 0 subtracts); see the refinement driver.
cudaError_t launch_krylov_update(cudaStream_t st, int64_t n, const double* base, const double* p, double* out,
                                 int sign, const Scalars* sc);
cudaError_t launch_krylov_direction(cudaStream_t st, int64_t n, const double* z, double* p, double beta_num,
                                    const Scalars* sc);

template <typename T>
cudaError_t launch_syrk_simt(cudaStream_t st, int64_t m, int64_t n, const T* A, const double* D, double* M64,
                             float* M32, int64_t ldm, const Scalars* sc);

// Blocked Cholesky in place; dinv (m) receives the reciprocals of the pivots.
template <typename T>
cudaError_t cholesky(cudaStream_t st, int64_t m, int64_t ldm, T* M, T* dinv, Scalars* sc);

// The single-launch tile Cholesky (chol_tiles.cu): 128 x 128 tiles; the task
// list comes from chol_tile_tasks (built once per m); state holds
// chol_tile_count(m)^2 ints; ticket is one counter.  Both are cleared here.
// Beyond 256 tile rows (m > 32768) the task list (~nb^3/6 tasks, built on
// the host at handle creation) grows past ~3M entries; such handles keep the
// multi-launch blocked factor.
constexpr int kTileCholMaxTiles = 256;
constexpr int kCholTile = 128;  // tile edge of the tile Cholesky and its triangular solves
int64_t chol_tile_count(int64_t m);
int chol_tiles_resident();  // resident CTAs on the current device, 0 on error
void chol_tile_tasks(int64_t m, int nproc, std::vector<int4>* out);
// Uinv receives U_l = L_ll^{-T} for every diagonal tile (nb x 128 x 128,
// row-major per tile), for trsv_lower_blk / trsv_upper_blk.
template <typename T>
cudaError_t cholesky_tiles(cudaStream_t st, int64_t m, int64_t ldm, T* M, T* dinv, T* Uinv, const int4* tasks,
                           int ntasks, int* state, unsigned* ticket, Scalars* sc, unsigned char* planes);
// Bytes of the BF16 operand planes of the FP32 tile factor (every tile below
// the diagonal, 96 KB each).
int64_t chol_plane_bytes(int64_t m);
// The double-float tile factor of the FP64 matrix M (FP64 tier of the mixed
// forms): M's lower triangle is turned into double-float pairs in place,
// factored by the tile Cholesky on the FP32 pipes (task list as the FP32
// factor's), and turned back into the FP64 factor L and FP64 pivot
// reciprocals dinv.  A pivot that is not positive sets PDAS_ERR_NOT_SPD.
cudaError_t cholesky_tiles_df(cudaStream_t st, int64_t m, int64_t ldm, double* M, double* dinv, const int4* tasks,
                              int ntasks, int* state, unsigned* ticket, Scalars* sc);
// The triangular solves with the FP32 tile factor (trsv_blk.cu).  The output
// (z, y) is the hand-off between blocks; it must not alias the input.
cudaError_t trsv_lower_blk(cudaStream_t st, int64_t m, int64_t ldm, const float* L, const float* Uinv,
                           const double* v, double* z, unsigned* ticket, Scalars* sc);
cudaError_t trsv_upper_blk(cudaStream_t st, int64_t m, int64_t ldm, const float* L, const float* Uinv,
                           const double* z, double* y, unsigned* ticket, Scalars* sc);
// scaled: the diagonal blocks are solved on pivot-scaled rows (the FP64 tier
// of the mixed forms, a preconditioner: shorter chains); else by plain
// substitution (the plain FP64 form's direct solve).
template <typename T>
cudaError_t trsv_lower(cudaStream_t st, int64_t m, int64_t ldm, const T* L, const T* dinv, const double* v,
                       double* z, int* flags, unsigned* tickets, Scalars* sc, bool scaled);
template <typename T>
cudaError_t trsv_upper_t(cudaStream_t st, int64_t m, int64_t ldm, const T* L, const T* dinv, const double* z,
                         double* y, int* flags, unsigned* tickets, Scalars* sc, bool scaled);

// sc->mnorm = max_p M[p][p] (before the factorization overwrites it).
template <typename T>
cudaError_t launch_diag_max(cudaStream_t st, int64_t m, int64_t ldm, const T* M, double* part, unsigned* tickets,
                            Scalars* sc);
// max_j |v_j| into sc->rho_norm (slot 1) or sc->dynorm (slot 2).
cudaError_t launch_absmax(cudaStream_t st, int64_t n, const double* v, double* part, unsigned* tickets, Scalars* sc,
                          int slot);

// Lower triangle of M64 = A D A' in double-float on the FP32 pipes (A exact
// in FP32: float or BF16 storage); D2 (n float2) receives D as hi + lo.
template <typename T>
cudaError_t launch_syrk_df(cudaStream_t st, int64_t m, int64_t n, const T* A, const double* D, float2* D2,
                           double* M64, int64_t ldm, const Scalars* sc);

// Akept (m x k, row-major) = the columns idx[0..k) of A; Dkept = D[idx].
template <typename T>
cudaError_t launch_gather_columns(cudaStream_t st, int64_t m, int64_t n, const T* A, const double* D, int64_t k,
                                  const int* idx, T* Akept, double* Dkept);

// Adjoint helpers: u = D .* g;  lb = D .* (w - g);  dA = -(la x' + y lb').
// out_p = (A D A')_pp without forming the matrix (m outputs).
template <typename T>
cudaError_t launch_normal_diag(cudaStream_t st, int64_t m, int64_t n, const T* A, const double* D, double* out,
                               const Scalars* sc);
cudaError_t launch_scale_vec(cudaStream_t st, int64_t n, const double* D, const double* g, double* u,
                             const Scalars* sc);
cudaError_t launch_adjoint_lb(cudaStream_t st, int64_t n, const double* D, const double* w, const double* g,
                              double* lb, const Scalars* sc);
// Refinement of the full adjoint system (see pdas_backward):
//   init:   lb = D (w - g), lc = -lb / x, wt = w
//   resid:  r1 = g - wt - s.*lc, r3 = -lb - x.*lc, t = D r1 - r3 - lb
//   update: db = D (w - r1) + r3, dc = (r3 - db) / x; lb += db, lc += dc, wt += w
cudaError_t launch_adjoint_init(cudaStream_t st, int64_t n, const double* D, const double* w, const double* g,
                                const double* x, double* lb, double* lc, double* wt, const Scalars* sc);
cudaError_t launch_adjoint_resid(cudaStream_t st, int64_t n, const double* D, const double* g, const double* x,
                                 const double* s, const double* wt, const double* lb, const double* lc, double* r1,
                                 double* r3, double* t, const Scalars* sc);
cudaError_t launch_adjoint_update(cudaStream_t st, int64_t n, const double* D, const double* w, const double* x,
                                  const double* r1, const double* r3, double* lb, double* lc, double* wt,
                                  const Scalars* sc);
cudaError_t launch_adjoint_dA(cudaStream_t st, int64_t m, int64_t n, const double* la, const double* x,
                              const double* y, const double* lb, double* dA, const Scalars* sc);

cudaError_t launch_convert_matrix(cudaStream_t st, int64_t m, int64_t ld_src, const void* src, int src_f64,
                                  int64_t ld_dst, void* dst, int dst_f64);

}  // namespace pdas
