// Error-path support: host-side fault injection and a self-test of the bounded grid barrier.
//
// Nothing here makes a GPU fault, trap or hang.  An injected allocation failure is raised on
// the host before cudaMallocAsync is called; an injected rank cap lowers the largest rank the
// persistent QR may reach, so that it stops short of the tolerance exactly as a real
// overflow would.  The barrier self-test runs the library's own grid barrier (gridsync.cuh)
// with one CTA that leaves before a barrier: the others wait for it only until a short limit,
// then return, and the host reports HBS_ERR_TIMEOUT as the solver's kernels do.
#include <atomic>
#include <mutex>
#include <string>

#include "devbuf.hpp"
#include "gridsync.cuh"
#include "profile.hpp"

namespace hbs {
namespace {
std::atomic<int64_t> g_alloc_countdown{-1};  // allocations left before the failing one (-1: off)
std::atomic<int> g_rank_cap{0};
}  // namespace

bool injected_alloc_failure() {
  int64_t v = g_alloc_countdown.load(std::memory_order_relaxed);
  while (v >= 0) {
    if (g_alloc_countdown.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return v == 0;
  }
  return false;
}

int injected_rank_cap() { return g_rank_cap.load(std::memory_order_relaxed); }

// Every CTA passes `rounds` barriers, except `absent` (if in range), which returns before the
// second.  A barrier that gives up returns -1 and the CTA leaves; the shared flag tells the host.
__global__ void k_barrier_selftest(GridSync* gs, int rounds, int absent, uint64_t limit_ns, int* passed) {
  for (int r = 0; r < rounds; ++r) {
    if (r == 1 && (int)blockIdx.x == absent) return;
    if (group_sync(gs, gridDim.x, limit_ns) != 0) return;
  }
  if (threadIdx.x == 0) atomicAdd(passed, 1);
}

}  // namespace hbs

extern "C" hbs_status hbs_fault_inject(int kind, int64_t value) {
  switch (kind) {
    case HBS_INJECT_CLEAR:
      hbs::g_alloc_countdown.store(-1);
      hbs::g_rank_cap.store(0);
      return HBS_OK;
    case HBS_INJECT_ALLOC_FAILURE:
      if (value < 0) break;
      hbs::g_alloc_countdown.store(value);
      return HBS_OK;
    case HBS_INJECT_RANK_CAP:
      if (value < 0 || value > (1 << 30)) break;
      hbs::g_rank_cap.store((int)value);
      return HBS_OK;
    default:
      break;
  }
  hbs::set_last_error("bad arguments to hbs_fault_inject");
  return HBS_ERR_INVALID_ARG;
}

extern "C" hbs_status hbs_barrier_selftest(int ctas, int absent_cta, double limit_s, int* passed, void* stream) {
  using namespace hbs;
  if (ctas < 1 || ctas > 64 || !(limit_s > 0.0) || limit_s > 10.0 || !passed) {
    set_last_error("bad arguments to hbs_barrier_selftest");
    return HBS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GridSync* gs = nullptr;
  int* dpassed = nullptr;
  hbs_status st = HBS_OK;
  try {
    HBS_CUDA(cudaMalloc(&gs, sizeof(GridSync)));
    HBS_CUDA(cudaMalloc(&dpassed, sizeof(int)));
    HBS_CUDA(cudaMemsetAsync(gs, 0, sizeof(GridSync), s));
    HBS_CUDA(cudaMemsetAsync(dpassed, 0, sizeof(int), s));
    int dev = 0, coop = 0, sms = 0;
    HBS_CUDA(cudaGetDevice(&dev));
    HBS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    HBS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (!coop || ctas > sms) throw Error(HBS_ERR_CUDA, "cooperative launch unavailable for the barrier self-test");
    GridSync* a0 = gs;
    int a1 = 3, a2 = absent_cta;
    uint64_t a3 = (uint64_t)(limit_s * 1e9);
    int* a4 = dpassed;
    void* args[] = {&a0, &a1, &a2, &a3, &a4};
    {
      std::lock_guard<std::mutex> lock(coop_mutex());
      prof::KScope _ks("k_barrier_selftest", s);
      HBS_CUDA(cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3(ctas), dim3(128), args, 0, s));
      HBS_LAUNCH_CHECK("k_barrier_selftest");
      HBS_CUDA(cudaStreamSynchronize(s));
    }
    GridSync hg{};
    HBS_CUDA(cudaMemcpy(&hg, gs, sizeof(GridSync), cudaMemcpyDeviceToHost));
    HBS_CUDA(cudaMemcpy(passed, dpassed, sizeof(int), cudaMemcpyDeviceToHost));
    if (hg.timed_out) {
      set_last_error("barrier self-test: a barrier wait gave up");
      st = HBS_ERR_TIMEOUT;
    }
  } catch (const Error& e) {
    set_last_error(e.what());
    st = e.code;
  }
  if (gs) cudaFree(gs);
  if (dpassed) cudaFree(dpassed);
  return st;
}
