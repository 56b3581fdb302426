// Device-side status word of one translation unit: kernels that give up a
// bounded wait (an mbarrier phase that never completed) set a bit here, besides
// the call-specific marker they leave in their outputs.  nk_query_status
// collects and clears the words of every translation unit (each includes this
// header once and defines its collector with NK_STATUS_COLLECTOR).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nk.h"

namespace nk {

// internal linkage: one word per translation unit (no relocatable device code)
static __device__ unsigned int g_dev_status = 0u;

__device__ __forceinline__ void dev_status_set(unsigned int bits) {
  atomicOr(&g_dev_status, bits);
}

// OR this unit's word into *out and clear it (one thread)
static __global__ void collect_status_kernel(int32_t* out) {
  const unsigned int v = atomicExch(&g_dev_status, 0u);
  if (v) atomicOr(reinterpret_cast<unsigned int*>(out), v);
}

}  // namespace nk

// Defines `nk_status name(int32_t* out, cudaStream_t st)` for this unit.
#define NK_STATUS_COLLECTOR(name)                                   \
  nk_status name(int32_t* out, cudaStream_t st) {                   \
    collect_status_kernel<<<1, 1, 0, st>>>(out);                    \
    return check_launch(#name);                                     \
  }
