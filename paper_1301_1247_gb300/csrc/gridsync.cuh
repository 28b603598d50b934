// Grid-wide barrier for persistent kernels launched with cudaLaunchCooperativeKernel
// (which guarantees that every CTA of the grid is resident at once).  Every wait is
// bounded: a CTA that waits longer than kGridWaitNs sets the shared timed-out flag and
// returns -1, and so do all CTAs that reach a barrier after that, so a persistent kernel
// always ends; the host reads the flag and reports HBS_ERR_TIMEOUT.
#pragma once

#include <cstdint>

namespace hbs {

struct __align__(128) GridSync {  // one cache line: the barriers of a batch share none
  unsigned int arrive;  // arrivals since the launch (count per completed barrier)
  int timed_out;
  int pad[30];
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int atom_add_acq_rel_u32(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

constexpr uint64_t kGridWaitNs = 2000000000ull;  // 2 s per barrier

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier over `count` CTAs sharing *gs (all of the grid, or the CTAs of one matrix of a
// batch; *gs zeroed before the launch).  The arrival counter only grows: the b-th barrier
// is complete once it reaches (b + 1) count, and each CTA learns b from the value its own
// arrival returns, so nothing is reset between barriers.  Returns 0, or -1 if a wait gave
// up (after limit_ns, or at once if another CTA already gave up).  Every one of the
// `count` CTAs must call it the same number of times.
__device__ __forceinline__ int group_sync(GridSync* gs, unsigned int count, uint64_t limit_ns = kGridWaitNs) {
  __shared__ int s_res;
  __syncthreads();  // the CTA's writes happen before thread 0's release below
  if (threadIdx.x == 0) {
    // release: this CTA's writes; acquire: those of the CTAs that arrived before it
    const unsigned int old = atom_add_acq_rel_u32(&gs->arrive, 1u);
    const unsigned int target = (old / count + 1u) * count;
    int ok = 0;
    if (old + 1u != target) {
      const uint64_t t0 = global_ns();
      unsigned int it = 0;
      while ((int)(ld_acquire_u32(&gs->arrive) - target) < 0) {
        if ((++it & 15u) == 0) {
          if (*(volatile int*)&gs->timed_out) { ok = -1; break; }
          if (global_ns() - t0 > limit_ns) {
            atomicExch(&gs->timed_out, 1);
            ok = -1;
            break;
          }
        }
        __nanosleep(32);
      }
    }
    s_res = ok;
  }
  __syncthreads();
  const int r = s_res;
  __syncthreads();
  return r;
}

__device__ __forceinline__ int grid_sync(GridSync* gs) { return group_sync(gs, gridDim.x); }

}  // namespace hbs
