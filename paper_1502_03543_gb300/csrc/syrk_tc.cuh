// syrk_tc.cuh -- the normal matrix M = A D A' (Section V) on the tcgen05
// tensor cores for the mixed-precision forms: operands staged by TMA, FP32
// accumulation in tensor memory, lower-triangle tiles only.
#pragma once

#include "pdas_internal.cuh"

namespace pdas {

struct TcWorkspace {
  int form = 0;         // PDAS_BF16_IR or PDAS_TF32_IR
  int a_dtype = 0;
  int splits = 0;       // low-precision terms of D.*A
  int64_t m = 0, n = 0;
  int64_t kpad = 0;     // n rounded up to the MMA K step
  int64_t mpad = 0;     // m rounded up to the tile edge
  void* opa = nullptr;  // A in the MMA type, mpad x kpad (TF32 form, or padded BF16)
  void* opb = nullptr;  // splits x mpad x kpad: the terms of D.*A
  void* host = nullptr; // host-side state (tensor maps, launch shape)
};

// Allocates the operand buffers; cudaErrorNotSupported if the tensor-core
// path is not built for this form.
cudaError_t tc_workspace_create(TcWorkspace* w, int form, int a_dtype, int splits, int64_t m, int64_t n);
void tc_workspace_destroy(TcWorkspace* w);

// Writes the split terms (D.*A)_t (and a padded copy of A if its rows are
// not 16-byte aligned).  *launches receives the kernels started.
cudaError_t tc_prepare(cudaStream_t st, TcWorkspace* w, const void* A, const double* D, int* launches);

// Lower triangle of M32 (leading dimension ldm) = sum over the split terms of
// A (D.*A)_t', FP32 accumulation (after tc_prepare).
cudaError_t tc_syrk(cudaStream_t st, TcWorkspace* w, const void* A, float* M32, int64_t ldm, const Scalars* sc,
                    int* launches);

}  // namespace pdas
