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

// Lower triangle of M32 (leading dimension ldm) = sum over the split terms of
// A (D.*A)_t', FP32 accumulation.  *launches receives the kernels started.
cudaError_t tc_form_normal(cudaStream_t st, TcWorkspace* w, int form, int a_dtype, const void* A, const double* D,
                           int64_t m, int64_t n, float* M32, int64_t ldm, const Scalars* sc, int* launches);

}  // namespace pdas
