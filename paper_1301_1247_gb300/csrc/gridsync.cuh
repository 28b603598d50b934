// Grid-wide barrier for persistent kernels launched with cudaLaunchCooperativeKernel
// (which guarantees that every CTA of the grid is resident at once).  Every wait is
// bounded: a CTA that waits longer than kGridWaitNs sets the shared timed-out flag and
// returns -1, and so do all CTAs that reach a barrier after that, so a persistent kernel
// always ends; the host reads the flag and reports HBS_ERR_TIMEOUT.
#pragma once

#include <cstdint>

namespace hbs {

struct __align__(128) GridSync {  // one cache line: the barriers of a batch share none
  unsigned int arrive;  // CTAs arrived in the current generation
  unsigned int gen;     // generation counter
  int timed_out;
  int pad;
  long long sum[2];     // per-generation (parity) sum of the CTAs' contributions
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

__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr uint64_t kGridWaitNs = 2000000000ull;  // 2 s per barrier

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier over `count` CTAs sharing *gs (all of the grid, or the CTAs of one matrix of a
// batch).  Returns the sum of `contrib` (taken from thread 0 of each CTA) over those CTAs
// for this generation, or -1 if a wait gave up.  Every one of them must call it the same
// number of times.
__device__ __forceinline__ long long group_sync_sum(GridSync* gs, long long contrib, unsigned int count) {
  __shared__ long long s_res;
  __syncthreads();  // the CTA's writes happen before thread 0's release below
  if (threadIdx.x == 0) {
    // gen cannot advance before this CTA arrives, so a relaxed read gives the current one
    const unsigned int g = *(volatile unsigned int*)&gs->gen;
    long long* slot = &gs->sum[g & 1u];
    if (contrib != 0) atomicAdd(reinterpret_cast<unsigned long long*>(slot), (unsigned long long)contrib);
    // release: this CTA's writes (and its contribution); acquire: those of earlier arrivals
    const unsigned int a = atom_add_acq_rel_u32(&gs->arrive, 1u);
    bool ok = true;
    if (a == count - 1) {
      // Every CTA has arrived, so the readers of the other parity's slot (previous
      // generation) are done with it: clear it for the next generation.
      gs->sum[(g + 1u) & 1u] = 0;
      gs->arrive = 0;
      st_release_u32(&gs->gen, g + 1u);  // publishes everything the arrivals released
    } else {
      const uint64_t t0 = global_ns();
      while (ld_acquire_u32(&gs->gen) == g) {
        if (*(volatile int*)&gs->timed_out) { ok = false; break; }
        if (global_ns() - t0 > kGridWaitNs) {
          atomicExch(&gs->timed_out, 1);
          ok = false;
          break;
        }
        __nanosleep(32);
      }
    }
    s_res = ok ? *(volatile long long*)slot : -1;
  }
  __syncthreads();
  const long long r = s_res;
  __syncthreads();
  return r;
}

__device__ __forceinline__ long long grid_sync_sum(GridSync* gs, long long contrib) {
  return group_sync_sum(gs, contrib, gridDim.x);
}

}  // namespace hbs
