// reduce_util.cuh -- deterministic block reductions shared by the
// bandwidth-bound kernels: every thread accumulates a fixed strided slice,
// blocks reduce with a fixed shuffle tree, and the last block to finish
// (ticket counter, no float atomics) combines the per-block partials in block
// order, so results are bit-identical from run to run.
#pragma once

#include "pdas_internal.cuh"

namespace pdas {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// op: 0 sum, 1 max, 2 min.  Result valid in thread 0.
template <int OP>
__device__ double block_reduce(double v, double* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = OP == 0 ? warp_sum(v) : OP == 1 ? warp_max(v) : warp_min(v);
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  double t = OP == 0 ? 0.0 : OP == 1 ? -INFINITY : INFINITY;
  if (w == 0) {
    if (lane < nw) t = sm[lane];
    t = OP == 0 ? warp_sum(t) : OP == 1 ? warp_max(t) : warp_min(t);
  }
  return t;
}

// True in every thread of the block that finishes last.  Partials written
// before the call are visible to that block.
__device__ bool last_block(unsigned* ticket) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1;
  __syncthreads();
  return last;
}

// Combine nparts partials in index order by one block (fixed order).
template <int OP>
__device__ double combine(const double* part, int nparts, double* sm) {
  double v = OP == 0 ? 0.0 : OP == 1 ? -INFINITY : INFINITY;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    double p = __ldcg(part + i);
    v = OP == 0 ? v + p : OP == 1 ? fmax(v, p) : fmin(v, p);
  }
  return block_reduce<OP>(v, sm);
}

__device__ __forceinline__ bool failed(const Scalars* sc) { return *(volatile const int*)&sc->status != 0; }

int grid_for(int64_t n, int per_thread = 1) {
  int64_t g = (n + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
  if (g < 1) g = 1;
  if (g > 1184) g = 1184;  // 8 blocks per SM on 148+ SMs; strided loops cover the rest
  return (int)g;
}

template <typename T>
bool vec_aligned(const T* A, int64_t n) {
  return ((uintptr_t)A % 16 == 0) && ((n * (int64_t)sizeof(T)) % 16 == 0);
}

}  // namespace

}  // namespace pdas
