// Bounded grid-wide barrier for cooperative launches (every CTA co-resident).
#pragma once
#include "common.cuh"

namespace ptk {

constexpr long long GRID_WAIT_LIMIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz

struct GridSync {
  unsigned* count;   // arrival counter, zeroed before each launch
  int* abort;        // raised by a CTA whose wait timed out; releases every other CTA
  long long limit;   // wait limit in clock cycles (GRID_WAIT_LIMIT_CYCLES for the path's kernels)
};

// Returns false when aborted (timeout here or elsewhere). The arrival counter only grows:
// barrier k of the launch is complete once it reaches k * gridDim.x, so one atomic per CTA and
// polling of the same word suffice. The abort flag and the time limit are checked every 64 polls;
// on expiry the CTA records ST_TIMEOUT and raises the abort flag.
__device__ __forceinline__ bool grid_barrier(const GridSync& gs, int* status) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned old = atomicAdd(gs.count, 1u);
    const unsigned target = (old / gridDim.x + 1u) * gridDim.x;
    volatile unsigned* vc = gs.count;
    const long long t0 = clock64();
    for (int it = 1;; ++it) {
      if ((int)(*vc - target) >= 0) break;
      if ((it & 63) == 0) {
        if (*(volatile int*)gs.abort) { ok = 0; break; }
        if (clock64() - t0 > gs.limit) {
          atomicOr(status, ST_TIMEOUT);
          atomicExch(gs.abort, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

}  // namespace ptk
