// syrk_tc.cu -- tensor-core normal-matrix builder (not built yet).
#include "syrk_tc.cuh"

namespace pdas {

cudaError_t tc_workspace_create(TcWorkspace* w, int form, int a_dtype, int splits, int64_t m, int64_t n) {
  (void)w; (void)form; (void)a_dtype; (void)splits; (void)m; (void)n;
  return cudaErrorNotSupported;
}

void tc_workspace_destroy(TcWorkspace* w) { (void)w; }

cudaError_t tc_form_normal(cudaStream_t st, TcWorkspace* w, int form, int a_dtype, const void* A, const double* D,
                           int64_t m, int64_t n, float* M32, int64_t ldm, const Scalars* sc, int* launches) {
  *launches = 0;
  (void)st; (void)w; (void)form; (void)a_dtype; (void)A; (void)D; (void)m; (void)n; (void)M32; (void)ldm; (void)sc;
  return cudaErrorNotSupported;
}

}  // namespace pdas
