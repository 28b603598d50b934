// Grid-wide barrier for persistent kernels launched with cudaLaunchCooperativeKernel
// (which guarantees that every CTA of the grid is resident at once).  Every wait is
// bounded: a CTA that waits longer than kGridWaitNs sets the shared timed-out flag and
// returns -1, and so do all CTAs that reach a barrier after that, so a persistent kernel
// always ends; the host reads the flag and reports HBS_ERR_TIMEOUT.
#pragma once

#include <cstdint>

namespace hbs {

struct GridSync {
  unsigned int arrive;  // CTAs arrived in the current generation
  unsigned int gen;     // generation counter
  int timed_out;
  int pad;
  long long sum[2];     // per-generation (parity) sum of the CTAs' contributions
};

constexpr uint64_t kGridWaitNs = 2000000000ull;  // 2 s per barrier

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier over all gridDim.x CTAs.  Returns the sum of `contrib` (taken from thread 0
// of each CTA) over the grid for this generation, or -1 if a wait gave up.  All CTAs
// must call it the same number of times.
__device__ __forceinline__ long long grid_sync_sum(GridSync* gs, long long contrib) {
  __shared__ long long s_res;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &gs->gen;
    const unsigned int g = *vgen;
    long long* slot = &gs->sum[g & 1u];
    if (contrib != 0) atomicAdd(reinterpret_cast<unsigned long long*>(slot), (unsigned long long)contrib);
    __threadfence();
    const unsigned int a = atomicAdd(&gs->arrive, 1u);
    bool ok = true;
    if (a == gridDim.x - 1) {
      // Every CTA has arrived, so the readers of the other parity's slot (previous
      // generation) are done with it: clear it for the next generation.
      gs->sum[(g + 1u) & 1u] = 0;
      gs->arrive = 0;
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (*vgen == g) {
        if (*(volatile int*)&gs->timed_out) { ok = false; break; }
        if (global_ns() - t0 > kGridWaitNs) {
          atomicExch(&gs->timed_out, 1);
          ok = false;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_res = ok ? *(volatile long long*)slot : -1;
  }
  __syncthreads();
  const long long r = s_res;
  __syncthreads();
  return r;
}

}  // namespace hbs
