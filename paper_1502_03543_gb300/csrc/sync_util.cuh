// sync_util.cuh -- inter-block signalling of the single-launch kernels (the
// triangular solves and the tile Cholesky): acquire/release flag accesses at
// GPU scope and bounded waits that record PDAS_ERR_TIMEOUT instead of
// spinning forever.
#pragma once

#include "pdas_internal.cuh"

namespace pdas {

__device__ __forceinline__ bool dev_failed(const Scalars* sc) { return *(volatile const int*)&sc->status != 0; }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s, unless the handle set its own limit

// The limit of one wait: sc->wait_us microseconds if the handle set a limit
// (pdas_set_wait_limit), else kWaitLimitNs.
__device__ __forceinline__ uint64_t wait_limit_ns(const Scalars* sc) {
  const int us = *(volatile const int*)&sc->wait_us;
  return us > 0 ? (uint64_t)us * 1000ull : kWaitLimitNs;
}

// One thread waits (bounded) until *p >= need.  Returns false if the device
// status is already an error or the limit passed (then PDAS_ERR_TIMEOUT is
// recorded).  The acquire orders the caller's later loads after the
// producer's release.
__device__ __forceinline__ bool wait_at_least(const int* p, int need, Scalars* sc) {
  if (ld_acquire(p) >= need) return true;
  const uint64_t t0 = global_ns(), limit = wait_limit_ns(sc);
  for (;;) {
    __nanosleep(64);
    if (ld_acquire(p) >= need) return true;
    if (dev_failed(sc)) return false;
    if (global_ns() - t0 > limit) {
      atomicCAS(&sc->status, 0, (int)PDAS_ERR_TIMEOUT);
      return false;
    }
  }
}

// Lane 0 of the calling warp waits (bounded) for flags[j] != 0; the warp
// learns the outcome.  The acquire by lane 0 and the warp barrier order the
// warp's later loads of the solution block after the producer's release.
__device__ inline bool warp_wait(const int* flags, int64_t j, Scalars* sc) {
  int res = 1;
  if ((threadIdx.x & 31) == 0) {
    const uint64_t t0 = global_ns(), limit = wait_limit_ns(sc);
    while (ld_acquire(flags + j) == 0) {
      if (dev_failed(sc)) { res = 0; break; }
      if (global_ns() - t0 > limit) {
        atomicCAS(&sc->status, 0, (int)PDAS_ERR_TIMEOUT);
        res = 0;
        break;
      }
      __nanosleep(32);
    }
  }
  res = __shfl_sync(0xffffffffu, res, 0);
  __syncwarp();
  return res != 0;
}

}  // namespace pdas
