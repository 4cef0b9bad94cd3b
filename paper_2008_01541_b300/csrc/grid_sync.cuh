// Bounded software grid barrier for kernels launched cooperatively (all CTAs
// co-resident).  The counter must be zero before the launch; barrier number b
// waits for the counter to reach gridDim.x * b.  Gives up after ~2^26 polls,
// records code 200 in status[1] and returns false.
#pragma once

namespace pdk {
__device__ inline bool grid_barrier(unsigned* ctr, unsigned target, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    atomicAdd(ctr, 1u);
    unsigned it = 0;
    while (*(volatile unsigned*)ctr < target) {
      if (++it > (1u << 26)) { ok = 0; atomicExch(status + 1, 200); break; }
      if (it > 64) __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}
}  // namespace pdk
