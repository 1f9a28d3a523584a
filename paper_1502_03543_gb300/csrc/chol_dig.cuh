// chol_dig.cuh -- the FP64 blocked Cholesky of the FP64 tier with its
// trailing updates on the tcgen05 tensor cores from exact fixed-point BF16
// digit planes (FP64-grade).
#pragma once

#include "pdas_internal.cuh"

namespace pdas {

// Smallest m whose FP64 tier takes this factor (below it the FP64 factor's
// SIMT updates are small and the double-float tile factor is as fast).
constexpr int64_t kCholDigMinM = 256;

struct CholDigWorkspace {
  int64_t m = 0;
  int64_t mpad = 0;        // m rounded up to 128
  int sub_partitions = 0;  // SM sub-partitions of the device (4 per SM): the row solve's launch shape
  void* planes = nullptr;  // 7 BF16 digit planes of mpad rows x 64 columns (the current panel)
  int* e = nullptr;        // row exponents of the current panel (mpad)
  void* host = nullptr;    // tensor maps
};

cudaError_t chol_dig_create(CholDigWorkspace* w, int64_t m);
void chol_dig_destroy(CholDigWorkspace* w);

// In place M = L L' (lower triangle, leading dimension ldm, m = w->m) in FP64
// by 64-column panels: the diagonal block's FP64 factor, the panel rows'
// FP64 solve and digits, then the trailing update on the tensor cores.  dinv (m) receives 1 / L_pp.  A pivot that is not
// positive sets PDAS_ERR_NOT_SPD (index in sc->fail_index).  *launches
// receives the kernels started.
cudaError_t cholesky_dig(cudaStream_t st, CholDigWorkspace* w, int64_t ldm, double* M, double* dinv, Scalars* sc,
                         int* launches);

}  // namespace pdas
