// Grid-wide barrier for cooperative launches (every block resident), with a
// bounded wait: used by the batched form's persistent plan and by the
// single-system distance sweeps.
#pragma once

#include <cstdint>

#include "dcm_internal.cuh"

namespace dcm {

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}


// Grid-wide barrier (arrival counter + generation).  Returns false, for the
// whole block, if the grid has been aborted or this block's wait ran past
// budget_ns (then it records DCM_ERR_TIMEOUT and raises the abort flag).
__device__ inline bool grid_sync(uint32_t* sync, uint32_t expected, int64_t budget_ns, int32_t* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* vs = sync;
    int good = vs[2] == 0;
    if (good) {
      const uint32_t gen = vs[1];
      __threadfence();
      if (atomicAdd(sync, 1u) + 1u == expected) {
        atomicExch(sync, 0u);
        __threadfence();
        atomicAdd(sync + 1, 1u);
      } else {
        // bounded twice: by the global nanosecond timer, and by a poll count
        // that a poll (an L2 round trip of well over 64 ns) cannot exhaust
        // before the time budget, in case the timer does not advance
        const uint64_t t0 = global_ns();
        const int64_t max_polls = budget_ns / 64 + 1024;
        int64_t polls = 0;
        while (vs[1] == gen) {
          if (vs[2] != 0) {
            good = 0;
            break;
          }
          if ((int64_t)(global_ns() - t0) > budget_ns || ++polls > max_polls) {
            good = 0;
            atomicExch(sync + 2, 1u);
            raise_status(status, DCM_ERR_TIMEOUT);
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}


}  // namespace dcm
