// syrk_dig.cuh -- the FP64 tier's normal matrix M = A D A' (Section V) on
// the tcgen05 tensor cores from fixed-point BF16 digit planes (A stored as
// BF16), exact products and exact sums: FP64-grade M.
#pragma once

#include "pdas_internal.cuh"

namespace pdas {

// Kept columns one call may take (this sizes the digit planes: 13 x m x
// 16384 BF16, 3.5 GB at m = 8192; more columns fall back to the
// double-float formation).
constexpr int64_t kDigMaxK = 16384;

struct DigWorkspace {
  int64_t m = 0;
  int64_t mpad = 0;         // m rounded up to 128
  int64_t kstride = 0;      // row stride of the digit planes (min(n, kDigMaxK) rounded up to 64)
  void* planes = nullptr;   // 13 BF16 planes of mpad x kstride: 5 digits of A, then 8 of D.*A
  int* ea = nullptr;        // row exponents of A (m)
  int* eb = nullptr;        // row exponents of D.*A (mpad)
  void* host = nullptr;     // tensor maps and the tile list
};

// Allocates the digit planes for m x n problems (kept columns up to
// min(n, kDigMaxK)) and builds the tensor maps and the tile list.
cudaError_t dig_workspace_create(DigWorkspace* w, int64_t m, int64_t n);
void dig_workspace_destroy(DigWorkspace* w);

// Lower triangle of M64 (leading dimension ldm) = A_K D_K A_K' over the k
// kept columns K = idx[0..k) of the m x n BF16 matrix A (idx null: the first
// k columns), k <= kstride.  Three launches (row exponents, digit planes,
// the tensor-core product); *launches receives the count.
cudaError_t dig_syrk(cudaStream_t st, DigWorkspace* w, const __nv_bfloat16* A, int64_t n, const double* D, int64_t k,
                     const int* idx, double* M64, int64_t ldm, Scalars* sc, int* launches);

}  // namespace pdas
