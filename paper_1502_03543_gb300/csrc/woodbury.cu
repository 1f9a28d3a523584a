// woodbury.cu -- the paper's own solver of the normal equations (Section V-A):
// (A D A') x = r through the Woodbury identity applied as n rank-one updates
// of A A', in the recurrence form of Egidi and Maponi.  For comparison with
// the Cholesky path; it costs O(m n^2) per solve against O(m^2 n) to form
// A D A'.  Entry points: include/pdas_woodbury.h.
//
// With U = A and V = A (D - I) (column l: u_l = a_l, v_l = (D_l - 1) a_l),
// A D A' = A A' + sum_l u_l v_l'.  From Y_0 = (A A')^{-1} A (columns y_{0,k})
// and x_0 = (A A')^{-1} r, step l = 1..n computes
//     den_l   = 1 + v_l' y_{l-1,l}
//     x_l     = x_{l-1}   - (v_l' x_{l-1}   / den_l) y_{l-1,l}
//     y_{l,k} = y_{l-1,k} - (v_l' y_{l-1,k} / den_l) y_{l-1,l},   k > l,
// and x_n solves the system.  Nothing in it depends on D before step 1, so
// A A', its factor and Y_0 are computed once per A (pdas_woodbury_prepare).
//
// Layout (the transposed storage the paper recommends, for coalescing): the
// columns y_k are the rows of an (n + 1) x m row-major array W, row n = x.
// Each step is one launch over the rows k > l (a warp per row: one dot
// product with v_l, one axpy with y_l), with v_l and y_l staged in shared
// memory per block; the warp of row l + 1 also forms den_{l+1} after its
// update.  No block waits on another: the launches order the steps.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "pdas_internal.cuh"
#include "pdas_woodbury.h"

struct pdas_wb_ctx {
  int64_t m = 0, n = 0, ldm = 0;
  int a_dtype = PDAS_A_F64;
  cudaStream_t st = nullptr;
  double* G = nullptr;      // A A' and its Cholesky factor, m x ldm
  double* ginv = nullptr;   // reciprocals of the factor's pivots (m)
  double* ones = nullptr;   // D = 1 for forming A A' (n)
  double* Y0 = nullptr;     // (A A')^{-1} A, transposed: n x m
  double* W = nullptr;      // working rows y_k (n) and x (row n): (n + 1) x m
  double* den = nullptr;    // den_l (n)
  pdas::Scalars* sc = nullptr;
  pdas::Scalars* sc_host = nullptr;  // pinned
  bool prepared = false;
  char errmsg[256] = {0};
};

namespace pdas {
namespace {

constexpr int kWbThreads = 256;  // 8 warps, a row of W each

template <typename T>
__device__ __forceinline__ double column_entry(const T* A, int64_t n, int64_t p, int64_t j) {
  return widen(A[p * n + j]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Rows of out (stride m): out_k = (L L')^{-1} b_k, one warp per right-hand
// side, by forward then back substitution with the factor L (lower, rows of
// stride ldm) and its pivot reciprocals.  b_k is column k of A (k < cols) or,
// for k == cols, the vector rhs.  The warp keeps its solution in its output
// row; each new entry needs the dot product of a row of L with the entries
// before it, summed across the warp in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kWbThreads) k_wb_solve_cols(int64_t m, int64_t n, int64_t ldm,
                                                              const double* __restrict__ L,
                                                              const double* __restrict__ dinv, const T* __restrict__ A,
                                                              int64_t cols, const double* __restrict__ rhs,
                                                              double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; k <= cols; k += warps) {
    if (k == cols && !rhs) break;
    double* z = out + k * m;
    for (int64_t i = 0; i < m; ++i) {  // L z = b
      const double* li = L + i * ldm;
      double acc = 0.0;
      for (int64_t j = lane; j < i; j += 32) acc = fma(li[j], z[j], acc);
      acc = warp_sum(acc);
      if (lane == 0) z[i] = ((k < cols ? column_entry(A, n, i, k) : rhs[i]) - acc) * dinv[i];
      __syncwarp();
    }
    for (int64_t i = m - 1; i >= 0; --i) {  // L' x = z
      double acc = 0.0;
      for (int64_t j = i + 1 + lane; j < m; j += 32) acc = fma(L[j * ldm + i], z[j], acc);
      acc = warp_sum(acc);
      if (lane == 0) z[i] = (z[i] - acc) * dinv[i];
      __syncwarp();
    }
  }
}

// den_0 = 1 + v_0' y_0 (one warp).
template <typename T>
__global__ void k_wb_first_den(int64_t m, int64_t n, const T* __restrict__ A, const double* __restrict__ D,
                               const double* __restrict__ W, double* __restrict__ den) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  double acc = 0.0;
  for (int64_t p = lane; p < m; p += 32) acc = fma(column_entry(A, n, p, 0), W[p], acc);
  acc = warp_sum(acc);
  if (lane == 0) den[0] = 1.0 + (D[0] - 1.0) * acc;
}

// Step l of the recurrence over rows k = l + 1 .. n of W (row n is x).
template <typename T>
__global__ void __launch_bounds__(kWbThreads) k_wb_step(int64_t m, int64_t n, int64_t l, const T* __restrict__ A,
                                                        const double* __restrict__ D, double* __restrict__ W,
                                                        double* __restrict__ den) {
  extern __shared__ double wb_smem[];
  double* vl = wb_smem;      // v_l = (D_l - 1) a_l
  double* yl = wb_smem + m;  // y_{l-1,l}, final since step l - 1
  const double dl = D[l] - 1.0;
  for (int64_t p = threadIdx.x; p < m; p += blockDim.x) {
    vl[p] = dl * column_entry(A, n, p, l);
    yl[p] = W[l * m + p];
  }
  __syncthreads();
  const double inv_den = 1.0 / den[l];
  const int lane = threadIdx.x & 31;
  const int64_t k = l + 1 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (k > n) return;
  double* wk = W + k * m;
  double acc = 0.0;
  for (int64_t p = lane; p < m; p += 32) acc = fma(vl[p], wk[p], acc);
  const double coef = warp_sum(acc) * inv_den;
  for (int64_t p = lane; p < m; p += 32) wk[p] = fma(-coef, yl[p], wk[p]);
  if (k == l + 1 && k < n) {  // den_{l+1} = 1 + v_{l+1}' y_{l,l+1} from the row just updated
    __syncwarp();
    const double dn = D[k] - 1.0;
    double a2 = 0.0;
    for (int64_t p = lane; p < m; p += 32) a2 = fma(column_entry(A, n, p, k), wk[p], a2);
    a2 = warp_sum(a2);
    if (lane == 0) den[k] = 1.0 + dn * a2;
  }
}

template <typename F>
cudaError_t with_a_dtype(int dt, F&& f) {
  switch (dt) {
    case PDAS_A_F64: return f((const double*)nullptr);
    case PDAS_A_F32: return f((const float*)nullptr);
    case PDAS_A_BF16: return f((const __nv_bfloat16*)nullptr);
  }
  return cudaErrorInvalidValue;
}

__global__ void k_fill(int64_t n, double v, double* out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = v;
}

unsigned solve_grid(int64_t warps) {
  return (unsigned)std::min<int64_t>((warps * 32 + kWbThreads - 1) / kWbThreads, 4736);
}

}  // namespace
}  // namespace pdas

using namespace pdas;

namespace {

pdas_status wb_fail(pdas_wb_ctx* h, cudaError_t e, const char* where) {
  snprintf(h->errmsg, sizeof(h->errmsg), "%s: %s", where, cudaGetErrorString(e));
  return PDAS_ERR_CUDA;
}
#define WCK(call)                                           \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return wb_fail(h, e_, #call);    \
  } while (0)

pdas_status wb_status(pdas_wb_ctx* h) {
  WCK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->st));
  WCK(cudaStreamSynchronize(h->st));
  return (pdas_status)h->sc_host->status;
}

}  // namespace

extern "C" {

pdas_status pdas_woodbury_create(int64_t m, int64_t n, int a_dtype, void* stream, pdas_wb_handle* out) {
  if (!out) return PDAS_ERR_ARG;
  *out = nullptr;
  if (m < 1 || n <= m || a_dtype < PDAS_A_F64 || a_dtype > PDAS_A_BF16) return PDAS_ERR_ARG;
  if (m > 14528) return PDAS_ERR_ARG;  // v_l and y_l, 2 m doubles, in one block's shared memory
  pdas_wb_ctx* h = new (std::nothrow) pdas_wb_ctx();
  if (!h) return PDAS_ERR_CUDA;
  h->m = m;
  h->n = n;
  h->ldm = (m + 15) / 16 * 16;
  h->a_dtype = a_dtype;
  h->st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  al((void**)&h->G, sizeof(double) * h->ldm * m);
  al((void**)&h->ginv, sizeof(double) * m);
  al((void**)&h->ones, sizeof(double) * n);
  al((void**)&h->Y0, sizeof(double) * n * m);
  al((void**)&h->W, sizeof(double) * (n + 1) * m);
  al((void**)&h->den, sizeof(double) * n);
  al((void**)&h->sc, sizeof(Scalars));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->sc_host, sizeof(Scalars));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_wb_step<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)(2 * m * sizeof(double)));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_wb_step<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)(2 * m * sizeof(double)));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_wb_step<__nv_bfloat16>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)(2 * m * sizeof(double)));
  if (e != cudaSuccess) {
    pdas_woodbury_destroy(h);
    return PDAS_ERR_CUDA;
  }
  *out = h;
  return PDAS_OK;
}

pdas_status pdas_woodbury_prepare(pdas_wb_handle h, const void* A) {
  if (!h || !A) return PDAS_ERR_ARG;
  h->prepared = false;
  WCK(cudaMemsetAsync(h->sc, 0, sizeof(Scalars), h->st));
  k_fill<<<(unsigned)std::min<int64_t>((h->n + 255) / 256, 1184), 256, 0, h->st>>>(h->n, 1.0, h->ones);
  WCK(cudaGetLastError());
  const cudaError_t pe = with_a_dtype(h->a_dtype, [&](auto tag) -> cudaError_t {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
    cudaError_t e = launch_syrk_simt<T>(h->st, h->m, h->n, (const T*)A, h->ones, h->G, nullptr, h->ldm, h->sc);
    if (e == cudaSuccess) e = cholesky<double>(h->st, h->m, h->ldm, h->G, h->ginv, h->sc);
    if (e != cudaSuccess) return e;
    k_wb_solve_cols<T><<<solve_grid(h->n), kWbThreads, 0, h->st>>>(h->m, h->n, h->ldm, h->G, h->ginv, (const T*)A,
                                                                  h->n, nullptr, h->Y0);
    return cudaGetLastError();
  });
  WCK(pe);
  pdas_status st = wb_status(h);
  h->prepared = st == PDAS_OK;
  return st;
}

pdas_status pdas_woodbury_solve(pdas_wb_handle h, const void* A, const double* D, const double* r, double* x,
                                double* min_den_out) {
  if (!h || !A || !D || !r || !x) return PDAS_ERR_ARG;
  if (!h->prepared) return PDAS_ERR_ARG;
  const int64_t m = h->m, n = h->n;
  WCK(cudaMemsetAsync(h->sc, 0, sizeof(Scalars), h->st));
  WCK(cudaMemcpyAsync(h->W, h->Y0, sizeof(double) * n * m, cudaMemcpyDeviceToDevice, h->st));
  const cudaError_t se = with_a_dtype(h->a_dtype, [&](auto tag) -> cudaError_t {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
    const T* At = (const T*)A;
    // x_0 = (A A')^{-1} r into row n (the rows k < n are Y_0 already)
    k_wb_solve_cols<T><<<1, 32, 0, h->st>>>(m, n, h->ldm, h->G, h->ginv, At, 0, r, h->W + n * m);
    k_wb_first_den<T><<<1, 32, 0, h->st>>>(m, n, At, D, h->W, h->den);
    cudaError_t e = cudaGetLastError();
    for (int64_t l = 0; l < n && e == cudaSuccess; ++l) {
      const int64_t rows = n - l;  // rows l + 1 .. n
      k_wb_step<T><<<(unsigned)((rows + kWbThreads / 32 - 1) / (kWbThreads / 32)), kWbThreads,
                     2 * m * sizeof(double), h->st>>>(m, n, l, At, D, h->W, h->den);
      e = cudaGetLastError();
    }
    return e;
  });
  WCK(se);
  WCK(cudaMemcpyAsync(x, h->W + n * m, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
  if (min_den_out) {
    std::vector<double> den((size_t)n);
    WCK(cudaMemcpyAsync(den.data(), h->den, sizeof(double) * n, cudaMemcpyDeviceToHost, h->st));
    WCK(cudaStreamSynchronize(h->st));
    double lo = HUGE_VAL;
    for (double d : den) lo = fmin(lo, fabs(d));
    *min_den_out = lo;
  }
  pdas_status st = wb_status(h);
  if (st != PDAS_OK) return st;
  return PDAS_OK;
}

void pdas_woodbury_destroy(pdas_wb_handle h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  double* bufs[] = {h->G, h->ginv, h->ones, h->Y0, h->W, h->den};
  for (double* p : bufs)
    if (p) cudaFree(p);
  if (h->sc) cudaFree(h->sc);
  if (h->sc_host) cudaFreeHost(h->sc_host);
  delete h;
}

const char* pdas_woodbury_last_error_message(pdas_wb_handle h) { return h ? h->errmsg : ""; }

}  // extern "C"
