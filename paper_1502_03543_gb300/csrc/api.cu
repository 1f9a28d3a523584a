// api.cu -- the C ABI of libpdas (include/pdas.h, include/pdas_components.h):
// handle life cycle, the per-iteration orchestration of the Newton-direction
// solve (Eq. 3 via Eq. 4, Section V), the psi ratio test and the step of the
// algorithm in Section III, and pdas_solve's outer loop.
//
// One iteration on the handle's stream (FP64 form):
//   scaling D = x/s -> r = A x -> M = A D A' (lower) -> Cholesky -> L z = r ->
//   L' dy = z -> w = A' dy, ds = -w, dx = D w - x -> psi, theta -> step, gap.
// Mixed forms replace the SYRK and Cholesky by their low-precision versions
// and refine dy in FP64 (refine()): the residual A x - A(D(A' dy)) is formed
// matrix-free in FP64 and corrected with the low-precision factor, as plain
// iterative refinement and, when that stalls, as conjugate gradients
// preconditioned by the same factor.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "pdas_internal.cuh"
#include "chol_dig.cuh"
#include "syrk_dig.cuh"
#include "syrk_tc.cuh"

using namespace pdas;

struct pdas_ctx {
  int64_t m = 0, n = 0, ldm = 0;
  pdas_options opt{};
  cudaStream_t st = nullptr;
  // FP64 vectors
  double *D = nullptr, *r = nullptr, *dy = nullptr, *dx = nullptr, *ds = nullptr, *w = nullptr, *u = nullptr;
  double *z = nullptr, *rho = nullptr, *delta = nullptr, *kp = nullptr, *kq = nullptr, *kz = nullptr;
  double* rd = nullptr;       // infeasible-start variant: dual residual c - A'y - s (n)
  double* part = nullptr;     // reduction partials (kPartMax)
  double* gt_part = nullptr;  // gemv_t partials, gt_chunks x n
  int gt_chunks = 1;
  int64_t gt_rows = 1;
  unsigned* tickets = nullptr;
  int* flags = nullptr;
  Scalars* sc = nullptr;
  Scalars* sc_host = nullptr;  // pinned
  int wait_us = 0;             // limit of the bounded inter-block waits (0: the 2 s default)
  int* wait_pinned = nullptr;  // pinned copy of wait_us, the source of its copy into sc
  double* M64 = nullptr;      // FP64 form; mixed forms: the FP64 tier's matrix (allocated at create)
  float* M32 = nullptr;
  double* dinv64 = nullptr;  // reciprocals of the pivots of the FP64 / FP32 factor
  float* dinv32 = nullptr;
  TcWorkspace tc{};
  DigWorkspace dig{};  // FP64 tier on the tensor cores (BF16 A): digit planes
  CholDigWorkspace cdig{};  // FP64 tier: the factor's trailing updates on the tensor cores
  int cur_f64 = 1;     // the workspace matrix in use is M64
  int refactored = 0;  // a mixed form switched to FP64 for good
  // column dropping for the FP64 factor of the mixed forms
  void* akept = nullptr;        // m x n elements of A's dtype (mixed forms with drop_tol > 0)
  double* dkept = nullptr;      // n
  int* kidx = nullptr;          // n
  std::vector<double> dhost;
  std::vector<int> idx_host;
  int64_t last_kept = 0;        // columns in the last FP64 factor of a mixed form
  bool no_drop_once = false;    // the dropped factor failed: use every column this time
  bool no_df_once = false;      // the double-float factor failed: form in FP64 this time
  float2* d2 = nullptr;         // D as FP32 pairs (double-float formation)
  int last_normal_form = 3;     // pdas_iter_info.normal_form of the last formation
  int last_factor_form = 3;     // pdas_iter_info.factor_form of the last factor
  bool have_factor = false;     // a factor from a previous step is in the workspace
  double* adj = nullptr;        // adjoint vectors (5 n + m)
  int4* chol_tasks = nullptr;   // task list of the tile Cholesky (FP32 factor)
  int chol_ntasks = 0;
  int* chol_state = nullptr;    // per-tile counters of the tile Cholesky
  float* uinv32 = nullptr;      // L_ll^{-T} of every diagonal tile of the FP32 tile factor
  unsigned char* chol_planes = nullptr;  // BF16 operand planes of the tile factor's off-diagonal tiles
  float2* pairs = nullptr;      // the vector of a double-float pass as FP32 pairs (max(m, n))
  int switch_reason = 0;  // pdas_iter_info.fp64_reason of that switch
  bool last_factor_df = false;    // the last factor was a fast FP64-tier factor (tensor-core or double-float)
  double last_rel_gap = HUGE_VAL;  // relative gap of the iterate after the last step
  bool no_dffactor_once = false;  // this iteration: that factor failed, use the FP64 factor
  int64_t err_index = -1;
  char errmsg[256] = {0};
  // diagnostics of the last direction
  int last_sweeps = 0;
  double last_resid = 0.0;
  int last_fp64 = 0;
  // profiling: event pairs around stages, and the kernel-launch count
  bool prof = false;
  std::vector<cudaEvent_t> evs;
  std::vector<int> ev_stage;  // per recorded pair: stage index
  size_t ev_used = 0;
  int open_stage = -1;
  double prof_ms[PDAS_STAGE_COUNT] = {0};
  int64_t prof_calls[PDAS_STAGE_COUNT] = {0};
  int64_t launches = 0;
};

namespace {

bool is_mixed(const pdas_ctx* h) { return h->opt.form != PDAS_FP64; }

pdas_status cuda_fail(pdas_ctx* h, cudaError_t e, const char* where) {
  snprintf(h->errmsg, sizeof(h->errmsg), "%s: %s", where, cudaGetErrorString(e));
  return PDAS_ERR_CUDA;
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);    \
  } while (0)

// A launch helper that starts `k` kernels: checked and counted.
#define KL(call, k)        \
  do {                     \
    CK(call);              \
    h->launches += (k);    \
  } while (0)

int64_t chol_launches(int64_t m) {
  int64_t k = 0;
  for (int64_t k0 = 0; k0 < m; k0 += kTile) k += (m - k0 - kTile > 0) ? 2 : 1;
  return k;
}

pdas_status prof_fold(pdas_ctx* h);

cudaError_t prof_record(pdas_ctx* h) {
  if (h->ev_used == h->evs.size()) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    h->evs.push_back(e);
  }
  return cudaEventRecord(h->evs[h->ev_used++], h->st);
}

pdas_status stage_begin(pdas_ctx* h, int stage) {
  if (!h->prof) return PDAS_OK;
  if (h->ev_used + 2 > 8192) {
    pdas_status s = prof_fold(h);
    if (s != PDAS_OK) return s;
  }
  CK(prof_record(h));
  h->open_stage = stage;
  return PDAS_OK;
}

pdas_status stage_end(pdas_ctx* h) {
  if (!h->prof || h->open_stage < 0) return PDAS_OK;
  CK(prof_record(h));
  h->ev_stage.push_back(h->open_stage);
  h->open_stage = -1;
  return PDAS_OK;
}

// Synchronise and add the recorded pairs to the accumulators.
pdas_status prof_fold(pdas_ctx* h) {
  CK(cudaStreamSynchronize(h->st));
  for (size_t i = 0; i < h->ev_stage.size(); ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->evs[2 * i], h->evs[2 * i + 1]));
    h->prof_ms[h->ev_stage[i]] += ms;
    h->prof_calls[h->ev_stage[i]] += 1;
  }
  h->ev_stage.clear();
  h->ev_used = 0;
  h->open_stage = -1;
  return PDAS_OK;
}

#define STAGE(h, k)                               \
  do {                                            \
    pdas_status s_ = stage_begin((h), (k));       \
    if (s_ != PDAS_OK) return s_;                 \
  } while (0)
#define STAGE_END(h)                              \
  do {                                            \
    pdas_status s_ = stage_end(h);                \
    if (s_ != PDAS_OK) return s_;                 \
  } while (0)

template <typename F>
pdas_status with_dtype(int dt, F&& f) {
  switch (dt) {
    case PDAS_A_F64: return f((const double*)nullptr);
    case PDAS_A_F32: return f((const float*)nullptr);
    case PDAS_A_BF16: return f((const __nv_bfloat16*)nullptr);
  }
  return PDAS_ERR_ARG;
}

// Reads the device scalars (one small copy + stream sync).
pdas_status read_scalars(pdas_ctx* h) {
  CK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return PDAS_OK;
}

pdas_status device_status(pdas_ctx* h) {
  const Scalars& s = *h->sc_host;
  if (s.status == PDAS_ERR_NOT_SPD) h->err_index = s.fail_index;
  return (pdas_status)s.status;
}

pdas_status reset_status(pdas_ctx* h) {
  CK(cudaMemsetAsync(h->sc, 0, sizeof(Scalars), h->st));
  if (h->wait_us > 0)  // a limit of the handle's own (pdas_set_wait_limit)
    CK(cudaMemcpyAsync(&h->sc->wait_us, h->wait_pinned, sizeof(int), cudaMemcpyHostToDevice, h->st));
  return PDAS_OK;
}

// A v -> out (base == null) or base - A v -> out; norm_slot as in launch_gemv.
// Double-float passes over A (gemv_df.cu) are available to the mixed forms
// when A is exact in FP32 (stored as FP32 or BF16) and exact_passes is off.
// The solve uses them only for the conjugate-gradient operator M p of the
// refinement while it factors in FP32: every quantity the acceptance test or
// the direction depends on
// (r = A x, the true residual r - A(D(A' dy)), w = A' dy) stays FP64, since
// the double-float rounding of a residual is close to the 1e-14 acceptance
// level, while in M p it scales with the search direction and only slows
// the iteration by rounding.  The component entry points pdas_gemv /
// pdas_gemv_t of a mixed handle expose the double-float pass itself.
bool df_passes(const pdas_ctx* h) { return is_mixed(h) && h->opt.a_dtype != PDAS_A_F64 && !h->opt.exact_passes; }

pdas_status gemv(pdas_ctx* h, const void* A, const double* v, const double* base, double* out, int norm_slot,
                 bool df = false) {
  if (df) {
    KL(launch_split_pairs(h->st, h->n, v, h->pairs), 1);
    if (h->opt.a_dtype == PDAS_A_F32)
      KL(launch_gemv_df<float>(h->st, h->m, h->n, (const float*)A, h->pairs, base, out, h->part, h->tickets, h->sc,
                               norm_slot), 1);
    else
      KL(launch_gemv_df<__nv_bfloat16>(h->st, h->m, h->n, (const __nv_bfloat16*)A, h->pairs, base, out, h->part,
                                       h->tickets, h->sc, norm_slot), 1);
    return PDAS_OK;
  }
  return with_dtype(h->opt.a_dtype, [&](auto tag) -> pdas_status {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
    KL(launch_gemv<T>(h->st, h->m, h->n, (const T*)A, v, base, out, h->part, h->tickets, h->sc, norm_slot), 1);
    return PDAS_OK;
  });
}

// w = A' u, then the finish mode (see launch_gemv_t_finish).
pdas_status gemv_t(pdas_ctx* h, const void* A, const double* u, int mode, const double* x, double* o0, double* o1,
                   double* o2, bool df = false, const double* rd = nullptr) {
  if (df) {
    KL(launch_split_pairs(h->st, h->m, u, h->pairs), 1);
    if (h->opt.a_dtype == PDAS_A_F32)
      KL(launch_gemv_t_df<float>(h->st, h->m, h->n, (const float*)A, h->pairs, h->gt_part, h->gt_chunks, h->gt_rows),
         1);
    else
      KL(launch_gemv_t_df<__nv_bfloat16>(h->st, h->m, h->n, (const __nv_bfloat16*)A, h->pairs, h->gt_part,
                                         h->gt_chunks, h->gt_rows), 1);
    KL(launch_gemv_t_finish(h->st, h->n, h->gt_chunks, h->gt_part, mode, x, h->D, o0, o1, o2, h->sc, rd), 1);
    return PDAS_OK;
  }
  pdas_status s = with_dtype(h->opt.a_dtype, [&](auto tag) -> pdas_status {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
    KL(launch_gemv_t<T>(h->st, h->m, h->n, (const T*)A, u, h->gt_part, h->gt_chunks, h->gt_rows), 1);
    return PDAS_OK;
  });
  if (s != PDAS_OK) return s;
  KL(launch_gemv_t_finish(h->st, h->n, h->gt_chunks, h->gt_part, mode, x, h->D, o0, o1, o2, h->sc, rd), 1);
  return PDAS_OK;
}

bool want_fp64(const pdas_ctx* h) { return !is_mixed(h) || h->refactored; }

size_t dtype_size(int dt) { return dt == PDAS_A_F64 ? 8 : dt == PDAS_A_F32 ? 4 : 2; }

// Columns for the FP64 factor of a mixed form: those with D_j >= drop_tol
// max D, at least drop_keep m of them (the largest D_j).  Returns the count
// (n = keep all; then idx is not built).
pdas_status select_columns(pdas_ctx* h, int64_t* kept) {
  const int64_t n = h->n;
  *kept = n;
  if (!(h->opt.drop_tol > 0) || h->no_drop_once) return PDAS_OK;
  h->dhost.resize(n);
  CK(cudaMemcpyAsync(h->dhost.data(), h->D, sizeof(double) * n, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  double dmax = 0.0;
  for (double d : h->dhost) dmax = std::max(dmax, d);
  double t = h->opt.drop_tol * dmax;
  int64_t count = 0;
  for (double d : h->dhost) count += d >= t;
  int64_t kmin = (int64_t)std::ceil(h->opt.drop_keep * (double)h->m);
  kmin = std::min(std::max<int64_t>(kmin, h->m), n);
  if (count < kmin) {  // lower the threshold to the kmin-th largest D
    std::vector<double> tmp(h->dhost);
    std::nth_element(tmp.begin(), tmp.begin() + (kmin - 1), tmp.end(), std::greater<double>());
    t = tmp[kmin - 1];
  }
  h->idx_host.clear();
  for (int64_t j = 0; j < n; ++j)
    if (h->dhost[j] >= t) h->idx_host.push_back((int)j);
  const int64_t k = (int64_t)h->idx_host.size();
  if (k >= n) return PDAS_OK;
  CK(cudaMemcpyAsync(h->kidx, h->idx_host.data(), sizeof(int) * k, cudaMemcpyHostToDevice, h->st));
  *kept = k;
  return PDAS_OK;
}

// a3: the normal matrix in the current precision.
pdas_status form_normal(pdas_ctx* h, const void* A) {
  if (want_fp64(h)) {
    pdas_status s;
    h->cur_f64 = 1;
    int64_t kept = h->n;
    if (is_mixed(h) && (s = select_columns(h, &kept)) != PDAS_OK) return s;
    h->last_kept = kept;
    // A mixed form whose A is exact in FP32 forms this matrix in double-float
    // on the FP32 pipes (FP64 remains the fallback when that factor fails).
    const bool df = is_mixed(h) && h->opt.a_dtype != PDAS_A_F64 && !h->no_df_once;
    // ... and, for BF16 A, on the tensor cores from exact fixed-point digit
    // planes (FP64-grade), when the kept columns fit the digit workspace
    const bool dig = df && h->opt.a_dtype == PDAS_A_BF16 && h->dig.planes && kept <= h->dig.kstride;
    h->last_normal_form = dig ? 4 : df ? 2 : 3;
    if (dig) {
      int kl = 0;
      CK(dig_syrk(h->st, &h->dig, (const __nv_bfloat16*)A, h->n, h->D, kept, kept < h->n ? h->kidx : nullptr,
                  h->M64, h->ldm, h->sc, &kl));
      h->launches += kl;
      return PDAS_OK;
    }
    return with_dtype(h->opt.a_dtype, [&](auto tag) -> pdas_status {
      using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
      const T* Aop = (const T*)A;
      const double* Dop = h->D;
      int64_t cols = h->n;
      if (kept < h->n) {
        KL(launch_gather_columns<T>(h->st, h->m, h->n, (const T*)A, h->D, kept, h->kidx, (T*)h->akept, h->dkept), 1);
        Aop = (const T*)h->akept;
        Dop = h->dkept;
        cols = kept;
      }
      if constexpr (std::is_same<T, double>::value) {
        KL(launch_syrk_simt<T>(h->st, h->m, cols, Aop, Dop, h->M64, nullptr, h->ldm, h->sc), 1);
      } else {
        if (df) KL(launch_syrk_df<T>(h->st, h->m, cols, Aop, Dop, h->d2, h->M64, h->ldm, h->sc), 2);
        else KL(launch_syrk_simt<T>(h->st, h->m, cols, Aop, Dop, h->M64, nullptr, h->ldm, h->sc), 1);
      }
      return PDAS_OK;
    });
  }
  h->cur_f64 = 0;
  h->last_normal_form = h->opt.form == PDAS_FP32_IR ? 1 : 0;
  if (h->opt.form == PDAS_FP32_IR) {
    return with_dtype(h->opt.a_dtype, [&](auto tag) -> pdas_status {
      using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
      KL(launch_syrk_simt<T>(h->st, h->m, h->n, (const T*)A, h->D, nullptr, h->M32, h->ldm, h->sc), 1);
      return PDAS_OK;
    });
  }
  int k = 0;
  if (h->prof && h->open_stage >= 0) h->open_stage = PDAS_STAGE_FOLD;  // the open interval starts the fold
  CK(tc_prepare(h->st, &h->tc, A, h->D, &k));
  h->launches += k;
  STAGE_END(h);
  STAGE(h, PDAS_STAGE_NORMAL);
  CK(tc_syrk(h->st, &h->tc, A, h->M32, h->ldm, h->sc, &k));
  h->launches += k;
  return PDAS_OK;
}

// The FP64 tier of a mixed form factors with the double-float tile factor
// (~3.5x faster than the FP64 factor on GB300's FP64 pipes) while the
// relative gap of the iterate exceeds opt.df_factor_floor, and with the FP64
// factor below it.  In the last iterations the forward error of the refined
// direction sets the gap that can be reached (the refinement accepts on a
// backward-error test), and a slightly different preconditioner there moved
// the gap-1e-8 run of the 8192 x 32768 problem from 54 iterations to 80.
pdas_status factor(pdas_ctx* h) {
  h->last_factor_df = false;
  if (h->cur_f64 && is_mixed(h) && h->cdig.planes && !h->no_dffactor_once) {
    // FP64 tier with fp64_tier_tc: the FP64 factor whose trailing updates run
    // on the tensor cores from exact digit planes (FP64-grade at every gap);
    // on a failed pivot the next attempt uses the FP64 SIMT factor
    h->last_factor_df = true;
    h->last_factor_form = 4;
    int k = 0;
    CK(cholesky_dig(h->st, &h->cdig, h->ldm, h->M64, h->dinv64, h->sc, &k));
    h->launches += k;
    return PDAS_OK;
  }
  if (h->cur_f64 && is_mixed(h) && h->chol_ntasks > 0 && !h->no_dffactor_once &&
      h->last_rel_gap > h->opt.df_factor_floor) {
    // FP64 tier of a mixed form: the double-float tile factor (FP32 pipes),
    // while the iterate is not yet close to the optimum
    h->last_factor_df = true;
    h->last_factor_form = 2;
    KL(cholesky_tiles_df(h->st, h->m, h->ldm, h->M64, h->dinv64, h->chol_tasks, h->chol_ntasks, h->chol_state,
                         h->tickets + T_CHOL, h->sc),
       4);
  } else if (h->cur_f64) {
    h->last_factor_form = 3;
    KL(cholesky<double>(h->st, h->m, h->ldm, h->M64, h->dinv64, h->sc), chol_launches(h->m));
  } else if (h->chol_ntasks == 0) {
    h->last_factor_form = 1;
    KL(cholesky<float>(h->st, h->m, h->ldm, h->M32, h->dinv32, h->sc), chol_launches(h->m));
  } else {
    h->last_factor_form = 0;
    KL(cholesky_tiles<float>(h->st, h->m, h->ldm, h->M32, h->dinv32, h->uinv32, h->chol_tasks, h->chol_ntasks,
                             h->chol_state, h->tickets + T_CHOL, h->sc, h->chol_planes),
       1);
  }
  return PDAS_OK;
}

// out = (L L')^{-1} rhs with the current factor (via h->z).
pdas_status factor_solve(pdas_ctx* h, const double* rhs, double* out) {
  if (h->cur_f64) {
    KL(trsv_lower<double>(h->st, h->m, h->ldm, h->M64, h->dinv64, rhs, h->z, h->flags, h->tickets, h->sc,
                          is_mixed(h)),
       1);
    KL(trsv_upper_t<double>(h->st, h->m, h->ldm, h->M64, h->dinv64, h->z, out, h->flags, h->tickets, h->sc,
                            is_mixed(h)),
       1);
  } else if (h->chol_ntasks > 0) {  // the tile factor, with the inverses of its diagonal tiles
    KL(trsv_lower_blk(h->st, h->m, h->ldm, h->M32, h->uinv32, rhs, h->z, h->tickets + T_TRSV, h->sc), 1);
    KL(trsv_upper_blk(h->st, h->m, h->ldm, h->M32, h->uinv32, h->z, out, h->tickets + T_TRSV, h->sc), 1);
  } else {
    KL(trsv_lower<float>(h->st, h->m, h->ldm, h->M32, h->dinv32, rhs, h->z, h->flags, h->tickets, h->sc, true), 1);
    KL(trsv_upper_t<float>(h->st, h->m, h->ldm, h->M32, h->dinv32, h->z, out, h->flags, h->tickets, h->sc, true),
       1);
  }
  return PDAS_OK;
}

// rho = r - A(D(A' v)); leaves w = A' v in h->w and ||rho||_inf in sc->rho_norm.
// df: by the double-float passes, for a residual that only starts the
// conjugate gradients (every residual that decides acceptance, and the w of
// an accepted direction, come from the FP64 passes).
pdas_status residual(pdas_ctx* h, const void* A, const double* v, bool df = false) {
  pdas_status s = gemv_t(h, A, v, 2, nullptr, h->u, nullptr, h->w, df);
  if (s != PDAS_OK) return s;
  return gemv(h, A, h->u, h->r, h->rho, 1, df);
}

// M v (matrix-free, FP64) -> out.
pdas_status apply_normal(pdas_ctx* h, const void* A, const double* v, double* out) {
  // (not once the solve has switched to an FP64 factor: there the FP64 factor
  // dominates the iteration, and near the end the operator's rounding decides
  // whether the refinement still reaches its tolerance)
  const bool df = df_passes(h) && !h->refactored;
  pdas_status s = gemv_t(h, A, v, 2, nullptr, h->u, nullptr, nullptr, df);
  if (s != PDAS_OK) return s;
  return gemv(h, A, h->u, nullptr, out, -1, df);
}

// FP64 refinement of dy for the mixed forms (a6): conjugate gradients on
// M dy = r with the factor as preconditioner, started from dy = (L L')^{-1} r.
// M is applied matrix-free in FP64 (A(D(A' v))), so the result is as
// accurate as FP64 arithmetic allows whatever the precision of the factor.
// The recurrence residual is confirmed against the true residual r - M dy
// before acceptance and every 10 steps (and replaces it when they differ).
// Accepted when ||r - M dy||_inf <= refine_tol ||r||_inf, or when the
// normwise backward error ||r - M dy||_inf / (max_p M_pp ||dy||_inf +
// ||r||_inf) <= refine_be.  On return h->w = A' dy of the final dy;
// *ok = 0 if neither test passed within refine_max steps.
pdas_status refine(pdas_ctx* h, const void* A, int* ok) {
  *ok = 0;
  const double tol = h->opt.refine_tol, be_tol = h->opt.refine_be;
  const int cap = h->opt.refine_max;
  pdas_status s;
  // With an FP32 factor the first residual is ~1e-7 of r and starts the
  // conjugate gradients: the double-float passes form it (two FP64 passes
  // saved per direction); a first residual that would be accepted is formed
  // again by the FP64 passes.
  const bool cheap_first = df_passes(h) && !h->cur_f64;
  auto true_residual = [&](bool df = false) -> pdas_status {
    pdas_status t = residual(h, A, h->dy, df);  // rho, ||rho||, w = A'dy
    if (t != PDAS_OK) return t;
    KL(launch_absmax(h->st, h->m, h->dy, h->part, h->tickets, h->sc, 2), 1);
    if ((t = read_scalars(h)) != PDAS_OK) return t;
    return device_status(h);
  };
  auto restart = [&](double* rz) -> pdas_status {  // z = P^{-1} rho, p = z, rz = rho'z
    pdas_status t = factor_solve(h, h->rho, h->kz);
    if (t != PDAS_OK) return t;
    CK(cudaMemcpyAsync(h->kp, h->kz, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, h->st));
    KL(launch_dot(h->st, h->m, h->rho, h->kz, h->part, h->tickets, h->sc, 0), 1);
    if ((t = read_scalars(h)) != PDAS_OK) return t;
    *rz = h->sc_host->dot_a;
    return device_status(h);
  };
  if ((s = true_residual(cheap_first)) != PDAS_OK) return s;
  const double rn = h->sc_host->rnorm > 0 ? h->sc_host->rnorm : 1.0;
  const double mn = h->sc_host->mnorm;
  auto accepted = [&](double res, double dyn) { return res <= tol * rn || res <= be_tol * (mn * dyn + rn); };
  double res = h->sc_host->rho_norm, dyn = h->sc_host->dynorm;
  if (cheap_first && accepted(res, dyn)) {  // acceptance is decided on the FP64 passes
    if ((s = true_residual()) != PDAS_OK) return s;
    res = h->sc_host->rho_norm;
    dyn = h->sc_host->dynorm;
  }
  int its = 0;
  if (accepted(res, dyn)) {
    *ok = 1;
  } else {
    double rz = 0.0;
    if ((s = restart(&rz)) != PDAS_OK) return s;
    while (its < cap && rz > 0.0 && isfinite(rz)) {
      if ((s = apply_normal(h, A, h->kp, h->kq)) != PDAS_OK) return s;                 // q = M p
      KL(launch_dot(h->st, h->m, h->kp, h->kq, h->part, h->tickets, h->sc, 1), 1);       // p'q
      KL(launch_krylov_update(h->st, h->m, h->dy, h->kp, h->dy, +1, h->sc), 1);          // dy += a p
      KL(launch_krylov_update(h->st, h->m, h->rho, h->kq, h->rho, -1, h->sc), 1);        // rho -= a q
      ++its;
      KL(launch_absmax(h->st, h->m, h->rho, h->part, h->tickets, h->sc, 1), 1);
      KL(launch_absmax(h->st, h->m, h->dy, h->part, h->tickets, h->sc, 2), 1);
      if ((s = factor_solve(h, h->rho, h->kz)) != PDAS_OK) return s;                    // z = P^{-1} rho
      KL(launch_dot(h->st, h->m, h->rho, h->kz, h->part, h->tickets, h->sc, 0), 1);      // new rho'z
      KL(launch_krylov_direction(h->st, h->m, h->kz, h->kp, rz, h->sc), 1);              // p = z + b p
      if ((s = read_scalars(h)) != PDAS_OK) return s;
      if ((s = device_status(h)) != PDAS_OK) return s;
      if (!(h->sc_host->dot_b > 0.0)) break;  // the preconditioned operator lost definiteness
      rz = h->sc_host->dot_a;
      res = h->sc_host->rho_norm;
      dyn = h->sc_host->dynorm;
      if (accepted(res, dyn) || its % 10 == 0 || its == cap) {
        if ((s = true_residual()) != PDAS_OK) return s;
        res = h->sc_host->rho_norm;
        dyn = h->sc_host->dynorm;
        if (accepted(res, dyn)) {
          *ok = 1;
          break;
        }
        if ((s = restart(&rz)) != PDAS_OK) return s;
      }
    }
  }
  h->last_sweeps = its;
  h->last_resid = res / rn;
  return PDAS_OK;
}

// The right-hand side of the normal equations at (x, s): D = x/s, then
// r = A x (a2; the paper's system, which assumes A x = b and A'y + s = c),
// or, for the infeasible-start variant (iv != null: y, b, c), the dual
// residual rd = c - A'y - s and r = b + A D rd.
struct Infeasible {
  const double *y, *b, *c;
};
pdas_status normal_rhs(pdas_ctx* h, const void* A, const double* x, const double* s, const Infeasible* iv) {
  pdas_status st;
  KL(launch_scaling(h->st, h->n, x, s, h->D, h->part, h->tickets, h->sc), 1);
  if (!iv) return gemv(h, A, x, nullptr, h->r, 0);  // r = A x
  if ((st = gemv_t(h, A, iv->y, 0, nullptr, h->w, nullptr, nullptr)) != PDAS_OK) return st;  // w = A'y
  KL(launch_dual_residual(h->st, h->n, iv->c, s, h->w, h->D, h->rd, h->u, h->sc), 1);     // rd, u = -D rd
  return gemv(h, A, h->u, iv->b, h->r, 0);                                                // r = b - A u
}

// One Newton direction at (x, s): fills h->D, h->r, h->dy, h->dx, h->ds (and
// h->rd for the infeasible-start variant, iv != null).
pdas_status direction(pdas_ctx* h, const void* A, const double* x, const double* s, const Infeasible* iv = nullptr) {
  pdas_status st;
  if ((st = reset_status(h)) != PDAS_OK) return st;
  const double* rd = iv ? h->rd : nullptr;
  STAGE(h, PDAS_STAGE_RHS);
  if ((st = normal_rhs(h, A, x, s, iv)) != PDAS_OK) return st;
  STAGE_END(h);
  if (is_mixed(h) && !h->refactored && h->opt.dspread_refactor > 0) {
    if ((st = read_scalars(h)) != PDAS_OK) return st;
    if ((st = device_status(h)) != PDAS_OK) return st;
    if (h->sc_host->dmax / h->sc_host->dmin > h->opt.dspread_refactor) {
      h->refactored = 1;
      h->switch_reason = 1;
    }
  }
  h->no_drop_once = false;
  h->no_df_once = false;
  h->no_dffactor_once = false;
  for (int attempt = 0; attempt < 5; ++attempt) {
    STAGE(h, PDAS_STAGE_NORMAL);
    if ((st = form_normal(h, A)) != PDAS_OK) return st;
    STAGE_END(h);
    if (is_mixed(h)) {  // max_p M_pp for the backward-error test of the refinement
      if (h->cur_f64) KL(launch_diag_max<double>(h->st, h->m, h->ldm, h->M64, h->part, h->tickets, h->sc), 1);
      else KL(launch_diag_max<float>(h->st, h->m, h->ldm, h->M32, h->part, h->tickets, h->sc), 1);
    }
    STAGE(h, PDAS_STAGE_FACTOR);
    if ((st = factor(h)) != PDAS_OK) return st;
    STAGE_END(h);
    h->have_factor = true;  // (a failed factor is reported below and retried)
    STAGE(h, PDAS_STAGE_SOLVE);
    if ((st = factor_solve(h, h->r, h->dy)) != PDAS_OK) return st;
    h->last_fp64 = h->cur_f64;
    if (!is_mixed(h)) {  // the plain FP64 form: the direct solve of Section V-A, unrefined
      STAGE_END(h);
      h->last_sweeps = 0;
      h->last_resid = 0.0;
      STAGE(h, PDAS_STAGE_DIR);
      if ((st = gemv_t(h, A, h->dy, 1, x, h->dx, h->ds, nullptr, false, rd)) != PDAS_OK) return st;  // a7
      STAGE_END(h);
      return PDAS_OK;
    }
    if ((st = read_scalars(h)) != PDAS_OK) return st;
    st = device_status(h);
    if (st == PDAS_ERR_NOT_SPD) {  // low-precision factor broke down: FP64 from now on
      STAGE_END(h);
      if (h->cur_f64) {
        if (h->last_factor_df) h->no_dffactor_once = true;        // the FP64 factor next
        else if (h->last_normal_form == 2 || h->last_normal_form == 4) h->no_df_once = true;  // form it in FP64 next
        else if (h->last_kept < h->n) h->no_drop_once = true;      // then from every column
        else return st;                                            // the whole FP64 matrix is not SPD
      }
      if (!h->refactored) h->switch_reason = 2;
      h->refactored = 1;
      if ((st = reset_status(h)) != PDAS_OK) return st;
      if ((st = normal_rhs(h, A, x, s, iv)) != PDAS_OK) return st;
      continue;
    }
    if (st != PDAS_OK) return st;
    int ok = 0;
    if ((st = refine(h, A, &ok)) != PDAS_OK) return st;
    STAGE_END(h);
    if (ok || h->cur_f64) {
      // w = A' dy of the accepted dy is in h->w: dx = D w - x, ds = -w.  (An
      // FP64 factor is the last tier: its refined direction is used as is.)
      STAGE(h, PDAS_STAGE_DIR);
      KL(launch_gemv_t_finish(h->st, h->n, 0, nullptr, 3, x, h->D, h->dx, h->ds, h->w, h->sc, rd), 1);
      STAGE_END(h);
      return PDAS_OK;
    }
    h->refactored = 1;  // refinement failed: re-form and re-factor in FP64
    h->switch_reason = 3;
  }
  return PDAS_ERR_NOT_SPD;
}

pdas_status check_vec_args(const void* A, const double* x, const double* s) {
  if (!A || !x || !s) return PDAS_ERR_ARG;
  return PDAS_OK;
}

void fill_info(pdas_ctx* h, pdas_iter_info* info, bool stepped) {
  if (!info) return;
  const Scalars& s = *h->sc_host;
  memset(info, 0, sizeof(*info));
  info->dmax = s.dmax;
  info->dmin = s.dmin;
  info->refine_sweeps = h->last_sweeps;
  info->refine_resid = h->last_resid;
  info->used_fp64 = h->last_fp64;
  info->fp64_reason = (h->last_fp64 && is_mixed(h)) ? h->switch_reason : 0;
  info->factor_columns = (h->last_fp64 && is_mixed(h)) ? h->last_kept : h->n;
  info->normal_form = h->last_normal_form;
  info->factor_form = h->last_factor_form;
  if (stepped) {
    info->psi = s.psi;
    info->theta = s.theta;
    info->rel_gap = s.rel_gap;
    info->cx = s.cx;
    info->by = s.by;
    info->xs = s.xs;
    if (h->opt.infeasible) {
      info->pres = s.pres;
      info->dres = s.dres;
    }
  }
}

}  // namespace

// ===========================================================================
extern "C" {

void pdas_default_options(pdas_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->form = PDAS_FP64;
  opt->a_dtype = PDAS_A_F64;
  opt->max_iter = 500;
  opt->refine_tol = 1e-14;
  opt->refine_max = 40;
  opt->refine_be = 1e-14;
  opt->drop_tol = 1e-10;
  opt->drop_keep = 1.25;
  opt->exact_passes = 0;
  opt->dspread_refactor = 0.0;
  opt->stream = nullptr;
  opt->splits = 0;
  opt->stall_theta = 1e-12;
  opt->stall_count = 5;
  opt->infeasible = 0;
  opt->fp64_tier_tc = 1;
  opt->df_factor_floor = 1e-6;
}

const char* pdas_status_str(pdas_status st) {
  switch (st) {
    case PDAS_OK: return "ok";
    case PDAS_OPTIMAL: return "optimal (relative gap below tol)";
    case PDAS_OPTIMAL_EXACT: return "optimal (psi <= 1, full step)";
    case PDAS_MAX_ITER: return "iteration cap reached";
    case PDAS_STALLED: return "stalled (step lengths below stall_theta)";
    case PDAS_ZERO_DIRECTION: return "zero direction";
    case PDAS_ERR_ARG: return "invalid argument";
    case PDAS_ERR_NOT_INTERIOR: return "iterate not interior (x > 0 and s > 0 required)";
    case PDAS_ERR_NOT_SPD: return "normal matrix not positive definite";
    case PDAS_ERR_NONFINITE: return "non-finite value in direction or ratio test";
    case PDAS_ERR_TIMEOUT: return "device-side wait timed out";
    case PDAS_ERR_CUDA: return "CUDA error";
    case PDAS_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

pdas_status pdas_create(int64_t m, int64_t n, const pdas_options* opt_in, pdas_handle* out) {
  if (!out) return PDAS_ERR_ARG;
  *out = nullptr;
  pdas_options opt;
  if (opt_in) opt = *opt_in;
  else pdas_default_options(&opt);
  if (m < 1 || n <= m || m > (int64_t)1 << 20 || n > (int64_t)1 << 31) return PDAS_ERR_ARG;
  if (opt.form < PDAS_FP64 || opt.form > PDAS_FP32_IR) return PDAS_ERR_ARG;
  if (opt.a_dtype < PDAS_A_F64 || opt.a_dtype > PDAS_A_BF16) return PDAS_ERR_ARG;
  if (opt.max_iter < 1 || opt.refine_max < 0 || !(opt.refine_tol > 0) || !(opt.refine_be >= 0) ||
      !(opt.drop_tol >= 0) || !(opt.drop_keep >= 1.0) || opt.splits < 0 || (opt.exact_passes & ~1) ||
      opt.splits > 3 || (opt.infeasible & ~1) ||
      opt.stall_count < 1 || !(opt.stall_theta >= 0) || (opt.fp64_tier_tc & ~1) ||
      !(opt.df_factor_floor >= 0))
    return PDAS_ERR_ARG;
  if (opt.form == PDAS_BF16_IR && opt.a_dtype != PDAS_A_BF16) return PDAS_ERR_UNSUPPORTED;
  // TF32 form: TF32 x 3 (splits 0 or 3) or one TF32 product (splits 1); FP64 or FP32 storage
  if (opt.form == PDAS_TF32_IR && (opt.a_dtype == PDAS_A_BF16 || opt.splits == 2)) return PDAS_ERR_UNSUPPORTED;
  pdas_ctx* h = new (std::nothrow) pdas_ctx();
  if (!h) return PDAS_ERR_CUDA;
  h->m = m;
  h->n = n;
  h->ldm = (m + 15) / 16 * 16;
  h->opt = opt;
  h->st = (cudaStream_t)opt.stream;
  // gemv_t decomposition: row chunks so that ~4 blocks per SM stream A
  {
    const int64_t target_chunks = 64;
    int64_t rows = (m + target_chunks - 1) / target_chunks;
    if (rows < 16) rows = 16;
    h->gt_rows = rows;
    h->gt_chunks = (int)((m + rows - 1) / rows);
  }
  const int64_t nblk = (m + kTile - 1) / kTile;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  al((void**)&h->D, sizeof(double) * n);
  al((void**)&h->dx, sizeof(double) * n);
  al((void**)&h->ds, sizeof(double) * n);
  al((void**)&h->w, sizeof(double) * n);
  al((void**)&h->u, sizeof(double) * n);
  al((void**)&h->r, sizeof(double) * m);
  al((void**)&h->dy, sizeof(double) * m);
  al((void**)&h->z, sizeof(double) * m);
  al((void**)&h->rho, sizeof(double) * m);
  al((void**)&h->delta, sizeof(double) * m);
  al((void**)&h->kp, sizeof(double) * m);
  al((void**)&h->kq, sizeof(double) * m);
  al((void**)&h->kz, sizeof(double) * m);
  if (opt.infeasible) al((void**)&h->rd, sizeof(double) * n);
  al((void**)&h->part, sizeof(double) * kPartMax * 4);
  al((void**)&h->gt_part, sizeof(double) * n * h->gt_chunks);
  al((void**)&h->tickets, sizeof(unsigned) * T_COUNT);
  al((void**)&h->flags, sizeof(int) * (nblk + 1));
  if (opt.form != PDAS_FP64 && opt.a_dtype != PDAS_A_F64) al((void**)&h->pairs, sizeof(float2) * n);  // n > m
  al((void**)&h->sc, sizeof(Scalars));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->sc_host, sizeof(Scalars));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->wait_pinned, sizeof(int));
  if (e == cudaSuccess) *h->wait_pinned = 0;
  al((void**)&h->adj, sizeof(double) * (5 * n + m));  // pdas_backward
  if (e == cudaSuccess) {
    // Every buffer of the FP64 tier of a mixed form is allocated here too, so
    // that a solve allocates nothing once it runs (an out-of-memory error
    // comes back from pdas_create, not from an iteration in mid-solve): the
    // FP64 matrix and its pivots, D as FP32 pairs for the double-float
    // formation, and the compact copy of the kept columns.
    al((void**)&h->M64, sizeof(double) * h->ldm * m);
    al((void**)&h->dinv64, sizeof(double) * m);
    if (opt.form != PDAS_FP64) {
      al((void**)&h->M32, sizeof(float) * h->ldm * m);
      al((void**)&h->dinv32, sizeof(float) * m);
      if (opt.a_dtype != PDAS_A_F64) al((void**)&h->d2, sizeof(float2) * n);
      if (opt.drop_tol > 0) {
        al((void**)&h->akept, dtype_size(opt.a_dtype) * m * n);
        al((void**)&h->dkept, sizeof(double) * n);
        al((void**)&h->kidx, sizeof(int) * n);
      }
    }
  }
  if (e == cudaSuccess && opt.form != PDAS_FP64 && chol_tile_count(m) <= kTileCholMaxTiles) {
    // the single-launch tile Cholesky of the FP32 factor
    std::vector<int4> tasks;
    const int workers = chol_tiles_resident();
    if (workers < 1) e = cudaErrorUnknown;
    chol_tile_tasks(m, workers, &tasks);
    const int64_t nb = chol_tile_count(m);
    h->chol_ntasks = (int)tasks.size();
    al((void**)&h->chol_tasks, sizeof(int4) * tasks.size());
    al((void**)&h->chol_state, sizeof(int) * nb * nb);
    al((void**)&h->uinv32, sizeof(float) * nb * kCholTile * kCholTile);
    if (nb > 1) al((void**)&h->chol_planes, (size_t)chol_plane_bytes(m));
    if (e == cudaSuccess)
      e = cudaMemcpy(h->chol_tasks, tasks.data(), sizeof(int4) * tasks.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && opt.form != PDAS_FP64 && opt.a_dtype == PDAS_A_BF16 && opt.fp64_tier_tc)
    e = dig_workspace_create(&h->dig, m, n);
  if (e == cudaSuccess && opt.form != PDAS_FP64 && opt.fp64_tier_tc && m > kCholDigMinM)
    e = chol_dig_create(&h->cdig, m);
  if (e == cudaSuccess && (opt.form == PDAS_BF16_IR || opt.form == PDAS_TF32_IR)) {
    e = tc_workspace_create(&h->tc, opt.form, opt.a_dtype, opt.splits, m, n);
    if (e == cudaErrorNotSupported) {
      cudaGetLastError();
      pdas_destroy(h);
      return PDAS_ERR_UNSUPPORTED;
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->tickets, 0, sizeof(unsigned) * T_COUNT, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->sc, 0, sizeof(Scalars), h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) {
    pdas_destroy(h);
    return PDAS_ERR_CUDA;
  }
  h->cur_f64 = opt.form == PDAS_FP64;
  *out = h;
  return PDAS_OK;
}

void pdas_destroy(pdas_handle h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  double* vecs[] = {h->D, h->r, h->dy, h->dx, h->ds, h->w, h->u, h->z, h->rho, h->delta, h->kp, h->kq, h->kz,
                    h->part, h->gt_part, h->M64, h->rd};
  for (double* p : vecs)
    if (p) cudaFree(p);
  if (h->M32) cudaFree(h->M32);
  if (h->akept) cudaFree(h->akept);
  if (h->dkept) cudaFree(h->dkept);
  if (h->kidx) cudaFree(h->kidx);
  if (h->d2) cudaFree(h->d2);
  if (h->adj) cudaFree(h->adj);
  if (h->chol_tasks) cudaFree(h->chol_tasks);
  if (h->chol_state) cudaFree(h->chol_state);
  if (h->uinv32) cudaFree(h->uinv32);
  if (h->chol_planes) cudaFree(h->chol_planes);
  if (h->pairs) cudaFree(h->pairs);
  if (h->dinv64) cudaFree(h->dinv64);
  if (h->dinv32) cudaFree(h->dinv32);
  if (h->tickets) cudaFree(h->tickets);
  if (h->flags) cudaFree(h->flags);
  if (h->sc) cudaFree(h->sc);
  if (h->sc_host) cudaFreeHost(h->sc_host);
  if (h->wait_pinned) cudaFreeHost(h->wait_pinned);
  tc_workspace_destroy(&h->tc);
  dig_workspace_destroy(&h->dig);
  chol_dig_destroy(&h->cdig);
  for (cudaEvent_t e : h->evs) cudaEventDestroy(e);
  delete h;
}

int64_t pdas_last_error_index(pdas_handle h) { return h ? h->err_index : -1; }

pdas_status pdas_set_wait_limit(pdas_handle h, int64_t microseconds) {
  if (!h || microseconds < 0 || microseconds > 2147483647) return PDAS_ERR_ARG;
  CK(cudaStreamSynchronize(h->st));  // no copy of the old value is still pending
  h->wait_us = (int)microseconds;
  *h->wait_pinned = (int)microseconds;
  return PDAS_OK;
}

const char* pdas_last_error_message(pdas_handle h) { return h ? h->errmsg : ""; }

pdas_status pdas_profile_enable(pdas_handle h, int enable) {
  if (!h) return PDAS_ERR_ARG;
  if (enable) {
    CK(cudaStreamSynchronize(h->st));
    h->ev_stage.clear();
    h->ev_used = 0;
    h->open_stage = -1;
    for (int i = 0; i < PDAS_STAGE_COUNT; ++i) {
      h->prof_ms[i] = 0.0;
      h->prof_calls[i] = 0;
    }
    h->launches = 0;
  }
  h->prof = enable != 0;
  return PDAS_OK;
}

pdas_status pdas_profile_read(pdas_handle h, pdas_profile* out) {
  if (!h || !out) return PDAS_ERR_ARG;
  pdas_status s = prof_fold(h);
  if (s != PDAS_OK) return s;
  for (int i = 0; i < PDAS_STAGE_COUNT; ++i) {
    out->ms[i] = h->prof_ms[i];
    out->calls[i] = h->prof_calls[i];
  }
  out->launches = h->launches;
  return PDAS_OK;
}

pdas_status pdas_direction(pdas_handle h, const void* A, const double* x, const double* s, double* dx, double* dy,
                           double* ds, pdas_iter_info* info) {
  if (!h || check_vec_args(A, x, s) != PDAS_OK || !dx || !dy || !ds) return PDAS_ERR_ARG;
  h->err_index = -1;
  pdas_status st = direction(h, A, x, s);
  if (st != PDAS_OK) return st;
  CK(cudaMemcpyAsync(dx, h->dx, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(ds, h->ds, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(dy, h->dy, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, h->st));
  if ((st = read_scalars(h)) != PDAS_OK) return st;
  st = device_status(h);
  fill_info(h, info, false);
  return st;
}

pdas_status pdas_direction_infeasible(pdas_handle h, const void* A, const double* b, const double* c,
                                      const double* x, const double* y, const double* s, double* dx, double* dy,
                                      double* ds, pdas_iter_info* info) {
  if (!h || check_vec_args(A, x, s) != PDAS_OK || !b || !c || !y || !dx || !dy || !ds) return PDAS_ERR_ARG;
  if (!h->opt.infeasible) return PDAS_ERR_ARG;
  h->err_index = -1;
  const Infeasible iv{y, b, c};
  pdas_status st = direction(h, A, x, s, &iv);
  if (st != PDAS_OK) return st;
  CK(cudaMemcpyAsync(dx, h->dx, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(ds, h->ds, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(dy, h->dy, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, h->st));
  if ((st = read_scalars(h)) != PDAS_OK) return st;
  st = device_status(h);
  fill_info(h, info, false);
  return st;
}

pdas_status pdas_step(pdas_handle h, const void* A, const double* b, const double* c, double* x, double* y,
                      double* s, double alpha, pdas_iter_info* info) {
  if (!h || check_vec_args(A, x, s) != PDAS_OK || !b || !c || !y) return PDAS_ERR_ARG;
  if (!(alpha > 0.0 && alpha < 1.0)) return PDAS_ERR_ARG;
  h->err_index = -1;
  const bool variant = h->opt.infeasible != 0;
  const Infeasible iv{y, b, c};
  pdas_status st = direction(h, A, x, s, variant ? &iv : nullptr);
  if (st != PDAS_OK) return st;
  STAGE(h, PDAS_STAGE_STEP);
  KL(launch_psi(h->st, h->n, x, s, h->dx, h->ds, alpha, h->part, h->tickets, h->sc, variant), 1);
  KL(launch_step(h->st, h->m, h->n, b, c, x, y, s, h->dx, h->dy, h->ds, h->part, h->tickets, h->sc), 1);
  if (variant) {  // residuals of the new iterate: b - A x and c - A'y - s
    if ((st = gemv(h, A, x, b, h->rho, -1)) != PDAS_OK) return st;
    if ((st = gemv_t(h, A, y, 0, nullptr, h->w, nullptr, nullptr)) != PDAS_OK) return st;
    KL(launch_residual_norms(h->st, h->m, h->n, b, h->rho, c, h->w, s, h->part, h->tickets, h->sc), 1);
  }
  STAGE_END(h);
  if ((st = read_scalars(h)) != PDAS_OK) return st;
  st = device_status(h);
  fill_info(h, info, st == PDAS_OK);
  if (st != PDAS_OK) return st;
  h->last_rel_gap = variant ? fmax(fabs(h->sc_host->rel_gap), fmax(h->sc_host->pres, h->sc_host->dres))
                            : h->sc_host->rel_gap;
  // a full step ends the paper's method at an optimum; the variant's never does
  return !variant && h->sc_host->psi <= 1.0 ? PDAS_OPTIMAL_EXACT : PDAS_OK;
}

pdas_status pdas_solve(pdas_handle h, const void* A, const double* b, const double* c, double* x, double* y,
                       double* s, double alpha, double tol, int* iters_out, double* rel_gap_out) {
  if (iters_out) *iters_out = 0;
  if (!h || check_vec_args(A, x, s) != PDAS_OK || !b || !c || !y) return PDAS_ERR_ARG;
  if (!(alpha > 0.0 && alpha < 1.0) || !(tol > 0.0)) return PDAS_ERR_ARG;
  h->err_index = -1;
  h->refactored = 0;
  h->switch_reason = 0;
  // interior check before anything is modified
  pdas_status st = reset_status(h);
  if (st != PDAS_OK) return st;
  KL(launch_scaling(h->st, h->n, x, s, h->D, h->part, h->tickets, h->sc), 1);
  if ((st = read_scalars(h)) != PDAS_OK) return st;
  if ((st = device_status(h)) != PDAS_OK) return st;
  int small = 0, k = 0;
  pdas_status result = PDAS_MAX_ITER;
  double gap = INFINITY;
  for (k = 0; k < h->opt.max_iter; ++k) {
    pdas_iter_info info;
    st = pdas_step(h, A, b, c, x, y, s, alpha, &info);
    if (st < 0) {
      result = st;
      break;
    }
    gap = info.rel_gap;
    if (st == PDAS_OPTIMAL_EXACT) {
      result = st;
      ++k;
      break;
    }
    const bool converged = h->opt.infeasible ? fabs(gap) < tol && info.pres < tol && info.dres < tol : gap < tol;
    if (converged) {
      result = PDAS_OPTIMAL;
      ++k;
      break;
    }
    small = info.theta < h->opt.stall_theta ? small + 1 : 0;
    if (small >= h->opt.stall_count) {
      result = PDAS_STALLED;
      ++k;
      break;
    }
  }
  if (iters_out) *iters_out = k;
  if (rel_gap_out) *rel_gap_out = gap;
  return result;
}

pdas_status pdas_backward(pdas_handle h, const void* A, const double* x, const double* y, const double* s,
                          const double* dL_dx, double* dL_dA, double* dL_db, double* dL_dc) {
  if (!h || check_vec_args(A, x, s) != PDAS_OK || !y || !dL_dx || !dL_db || !dL_dc) return PDAS_ERR_ARG;
  if (!h->have_factor) return PDAS_ERR_ARG;  // the preconditioner comes from a previous step
  h->err_index = -1;
  const int64_t m = h->m, n = h->n;
  pdas_status st = reset_status(h);
  if (st != PDAS_OK) return st;
  double* lb = h->adj;      // dL/dc
  double* lc = lb + n;      // multiplier of X s = sigma
  double* wt = lc + n;      // A' la
  double* r1 = wt + n;      // residual of A' la + S lc = g
  double* r3 = r1 + n;      // residual of lb + X lc = 0
  double* la = r3 + n;      // dL/db (m)
  // The preconditioner is the factor of the previous iterate's D: allow the
  // conjugate gradients four times the usual number of steps.
  const int cap = h->opt.refine_max;
  auto solve_normal = [&](int* ok) -> pdas_status {  // (A D A') dy = h->r, w = A' dy
    pdas_status t = factor_solve(h, h->r, h->dy);
    if (t != PDAS_OK) return t;
    h->opt.refine_max = 4 * cap;
    t = refine(h, A, ok);
    h->opt.refine_max = cap;
    return t;
  };
  KL(launch_scaling(h->st, n, x, s, h->D, h->part, h->tickets, h->sc), 1);
  // max_p M_pp at this D for the backward-error test of the refinement (the
  // matrix itself is not formed: the preconditioner is the last factor);
  // ldm = 0 makes the diagonal reduction read the m-vector M_pp.
  st = with_dtype(h->opt.a_dtype, [&](auto tag) -> pdas_status {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
    KL(launch_normal_diag<T>(h->st, m, n, (const T*)A, h->D, h->kq, h->sc), 1);
    return PDAS_OK;
  });
  if (st != PDAS_OK) return st;
  KL(launch_diag_max<double>(h->st, m, 0, h->kq, h->part, h->tickets, h->sc), 1);
  // reduced solve: (A D A') la = A (D g); lb = D (A' la - g); lc = -lb / x
  KL(launch_scale_vec(h->st, n, h->D, dL_dx, h->u, h->sc), 1);
  if ((st = gemv(h, A, h->u, nullptr, h->r, 0)) != PDAS_OK) return st;
  int ok = 0;
  if ((st = solve_normal(&ok)) != PDAS_OK) return st;
  if (!ok) return PDAS_ERR_NOT_SPD;
  CK(cudaMemcpyAsync(la, h->dy, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
  KL(launch_adjoint_init(h->st, n, h->D, h->w, dL_dx, x, lb, lc, wt, h->sc), 1);
  // lb = D (A' la - g) cancels where D is large; two steps of refinement on
  // the full adjoint system [A' 0 S; 0 A 0; 0 I X] (la, lb, lc) = (g, 0, 0)
  // with FP64 residuals recover it.  Each correction solves the same
  // normal equations: (A D A') da = A (D r1 - r3 - lb).
  for (int it = 0; it < 2; ++it) {
    KL(launch_adjoint_resid(h->st, n, h->D, dL_dx, x, s, wt, lb, lc, r1, r3, h->u, h->sc), 1);
    if ((st = gemv(h, A, h->u, nullptr, h->r, 0)) != PDAS_OK) return st;
    if ((st = solve_normal(&ok)) != PDAS_OK) return st;
    if (!ok) break;  // the correction is at the rounding level: keep what we have
    KL(launch_axpy(h->st, m, 1.0, h->dy, la, h->sc), 1);
    KL(launch_adjoint_update(h->st, n, h->D, h->w, x, r1, r3, lb, lc, wt, h->sc), 1);
  }
  CK(cudaMemcpyAsync(dL_db, la, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(dL_dc, lb, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
  if (dL_dA) KL(launch_adjoint_dA(h->st, m, n, la, x, y, lb, dL_dA, h->sc), 1);
  if ((st = read_scalars(h)) != PDAS_OK) return st;
  return device_status(h);
}

// ---- components ------------------------------------------------------------
pdas_status pdas_form_normal(pdas_handle h, const void* A, const double* x, const double* s) {
  if (!h || check_vec_args(A, x, s) != PDAS_OK) return PDAS_ERR_ARG;
  pdas_status st = reset_status(h);
  if (st != PDAS_OK) return st;
  KL(launch_scaling(h->st, h->n, x, s, h->D, h->part, h->tickets, h->sc), 1);
  STAGE(h, PDAS_STAGE_NORMAL);
  if ((st = form_normal(h, A)) != PDAS_OK) return st;
  STAGE_END(h);
  if ((st = read_scalars(h)) != PDAS_OK) return st;
  return device_status(h);
}

pdas_status pdas_copy_matrix(pdas_handle h, void* dst, int* dtype_out) {
  if (!h || !dst) return PDAS_ERR_ARG;
  const size_t es = h->cur_f64 ? sizeof(double) : sizeof(float);
  const void* src = h->cur_f64 ? (const void*)h->M64 : (const void*)h->M32;
  if (!src) return PDAS_ERR_ARG;
  CK(cudaMemcpy2DAsync(dst, es * h->m, src, es * h->ldm, es * h->m, h->m, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (dtype_out) *dtype_out = h->cur_f64 ? PDAS_A_F64 : PDAS_A_F32;
  return PDAS_OK;
}

pdas_status pdas_load_matrix(pdas_handle h, const void* src, int dtype) {
  if (!h || !src || (dtype != PDAS_A_F64 && dtype != PDAS_A_F32)) return PDAS_ERR_ARG;
  if (!h->cur_f64 && !h->M32) return PDAS_ERR_ARG;
  void* dst = h->cur_f64 ? (void*)h->M64 : (void*)h->M32;
  if (!dst) return PDAS_ERR_ARG;
  KL(launch_convert_matrix(h->st, h->m, h->m, src, dtype == PDAS_A_F64, h->ldm, dst, h->cur_f64), 1);
  CK(cudaStreamSynchronize(h->st));
  return PDAS_OK;
}

pdas_status pdas_factor(pdas_handle h) {
  if (!h) return PDAS_ERR_ARG;
  h->err_index = -1;
  pdas_status st = reset_status(h);
  if (st != PDAS_OK) return st;
  if ((st = factor(h)) != PDAS_OK) return st;
  if ((st = read_scalars(h)) != PDAS_OK) return st;
  st = device_status(h);
  h->have_factor = st == PDAS_OK;
  return st;
}

pdas_status pdas_factor_solve(pdas_handle h, const double* rhs, double* out) {
  if (!h || !rhs || !out) return PDAS_ERR_ARG;
  pdas_status st = reset_status(h);
  if (st != PDAS_OK) return st;
  if ((st = factor_solve(h, rhs, h->delta)) != PDAS_OK) return st;
  CK(cudaMemcpyAsync(out, h->delta, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, h->st));
  if ((st = read_scalars(h)) != PDAS_OK) return st;
  return device_status(h);
}

pdas_status pdas_gemv(pdas_handle h, const void* A, const double* v, double* out) {
  if (!h || !A || !v || !out) return PDAS_ERR_ARG;
  pdas_status st = reset_status(h);
  if (st != PDAS_OK) return st;
  if ((st = gemv(h, A, v, nullptr, out, -1, df_passes(h))) != PDAS_OK) return st;
  if ((st = read_scalars(h)) != PDAS_OK) return st;
  return device_status(h);
}

pdas_status pdas_gemv_t(pdas_handle h, const void* A, const double* u, double* out) {
  if (!h || !A || !u || !out) return PDAS_ERR_ARG;
  pdas_status st = reset_status(h);
  if (st != PDAS_OK) return st;
  if ((st = gemv_t(h, A, u, 0, nullptr, out, nullptr, nullptr, df_passes(h))) != PDAS_OK) return st;
  if ((st = read_scalars(h)) != PDAS_OK) return st;
  return device_status(h);
}

}  // extern "C"
