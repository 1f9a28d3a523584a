// noalloc.cu -- out = A' u without a handle and without allocating device
// memory: pdas_gemv_t_noalloc (include/pdas_components.h).
//
// Who needs it: callers that cannot call cudaMalloc.  Examples are code that
// runs while someone else is capturing the stream into a CUDA graph
// (allocation is not a capturable operation), processes whose device memory
// belongs to another framework's pool that must not be bypassed, and
// real-time loops that forbid allocation after start-up.  A libpdas handle
// allocates its workspace in pdas_create, so those callers cannot use
// pdas_gemv_t; this entry point gives them the same product.
//
// The A' u kernel needs scratch for its per-row-chunk partial column sums.
// Here that scratch is one file-scope device array of fixed size,
// kNoallocBytes (PDAS_NOALLOC_SCRATCH_BYTES): a status block (cleared on
// every call) followed by the partials.  Every GPU that loads libpdas holds
// the array until the process exits.  All calls share it and it keeps the
// last call's contents, so calls that overlap on the GPU (different streams,
// or different host threads) race on it: serialise them.
//
// Host code cannot pass g_noalloc_scratch to a kernel directly -- in host
// code that name is a host-side stand-in, not a device address.  The device
// address is fetched once per device with cudaGetSymbolAddress, with that
// device current, on the first call made on it.  That first call also loads
// the kernels' module, so make it before any stream capture.  The address is
// kept for the life of the process: after cudaDeviceReset (which unloads the
// module and frees the array) it would be stale, so a process that resets a
// device must not call this entry point on that device again.
#include <mutex>

#include "pdas_internal.cuh"

namespace {

constexpr size_t kNoallocBytes = PDAS_NOALLOC_SCRATCH_BYTES;
constexpr size_t kStatusBytes = 256;  // Scalars block, then the partials
static_assert(sizeof(pdas::Scalars) <= kStatusBytes, "status block too small");
constexpr int64_t kPartialDoubles = (int64_t)((kNoallocBytes - kStatusBytes) / sizeof(double));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_device_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (set up once).
pdas_status scratch_on_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PDAS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return PDAS_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_device_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PDAS_ERR_CUDA;
    g_device_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_device_ptr[dev];
  return PDAS_OK;
}

template <typename T>
cudaError_t run(cudaStream_t st, int64_t m, int64_t n, const void* A, const double* u, double* out,
                unsigned char* base) {
  // The row-chunk split of the handle's pdas_gemv_t (chunks of at least 16
  // rows, at most 64 chunks), coarsened when the partials would not fit.
  int64_t rows = (m + 63) / 64;
  if (rows < 16) rows = 16;
  int64_t chunks = (m + rows - 1) / rows;
  const int64_t max_chunks = kPartialDoubles / n;
  if (chunks > max_chunks) {
    rows = (m + max_chunks - 1) / max_chunks;
    chunks = (m + rows - 1) / rows;
  }
  pdas::Scalars* sc = reinterpret_cast<pdas::Scalars*>(base);
  double* part = reinterpret_cast<double*>(base + kStatusBytes);
  cudaError_t e = cudaMemsetAsync(sc, 0, sizeof(pdas::Scalars), st);  // status must start at zero
  if (e != cudaSuccess) return e;
  e = pdas::launch_gemv_t<T>(st, m, n, static_cast<const T*>(A), u, part, (int)chunks, rows);
  if (e != cudaSuccess) return e;
  return pdas::launch_gemv_t_finish(st, n, (int)chunks, part, 0, nullptr, nullptr, out, nullptr, nullptr, sc);
}

}  // namespace

extern "C" pdas_status pdas_gemv_t_noalloc(int64_t m, int64_t n, int a_dtype, const void* A, const double* u,
                                           double* out, void* stream) {
  if (m < 1 || n < 1 || !A || !u || !out) return PDAS_ERR_ARG;
  if (n > kPartialDoubles) return PDAS_ERR_ARG;  // one chunk of partials must fit the scratch
  unsigned char* base = nullptr;
  pdas_status s = scratch_on_current_device(&base);
  if (s != PDAS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (a_dtype) {
    case PDAS_A_F64: e = run<double>(st, m, n, A, u, out, base); break;
    case PDAS_A_F32: e = run<float>(st, m, n, A, u, out, base); break;
    case PDAS_A_BF16: e = run<__nv_bfloat16>(st, m, n, A, u, out, base); break;
    default: return PDAS_ERR_ARG;
  }
  return e == cudaSuccess ? PDAS_OK : PDAS_ERR_CUDA;
}
