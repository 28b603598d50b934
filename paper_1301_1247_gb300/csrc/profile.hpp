// Launch accounting and optional CUDA-event timing of the library's kernels.
//
// Every kernel launch of the library goes through a KScope, which counts it; when
// profiling is enabled (hbs_profile_enable) the scope also records a CUDA event pair
// on the launching stream so that per-kernel device time, launches and the kernel's
// algorithmic flops and bytes can be read back with hbs_profile_get.  Each launch is also
// charged to the innermost named phase open on the launching host thread, so a phase's
// device time can be split by kernel.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cstdint>
#include <string>

namespace hbs {
namespace prof {

extern std::atomic<int64_t> g_launches;
extern std::atomic<int> g_enabled;

void record(const char* name, const char* phase, cudaStream_t s, cudaEvent_t a, cudaEvent_t b, double flops,
            double bytes, std::chrono::steady_clock::time_point issued);
// Add algorithmic work to a kernel's record when it is only known after the launch.
void add_work(const char* name, double flops, double bytes);
// Host wall time of a named phase (recorded only while profiling is enabled).
void host_phase(const char* name, double seconds);
cudaEvent_t new_event();

// The innermost phase open on this host thread (nullptr outside any phase).
inline const char*& current_phase() {
  static thread_local const char* p = nullptr;
  return p;
}

struct KScope {
  const char* name;
  cudaStream_t s;
  double flops, bytes;
  cudaEvent_t a = nullptr;
  const char* phase = nullptr;
  std::chrono::steady_clock::time_point issued;
  KScope(const char* n, cudaStream_t st, double fl = 0.0, double by = 0.0) : name(n), s(st), flops(fl), bytes(by) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_enabled.load(std::memory_order_relaxed)) {
      phase = current_phase();
      issued = std::chrono::steady_clock::now();
      a = new_event();
      cudaEventRecord(a, s);
    }
  }
  ~KScope() {
    if (a) {
      cudaEvent_t b = new_event();
      cudaEventRecord(b, s);
      record(name, phase, s, a, b, flops, bytes, issued);
    }
  }
};

// Host wall time of a block of work (synchronizes the stream at the end, only when
// profiling is enabled).
struct Phase {
  const char* name;
  cudaStream_t s;
  std::chrono::steady_clock::time_point t0;
  const char* outer;
  Phase(const char* n, cudaStream_t st) : name(n), s(st), t0(std::chrono::steady_clock::now()), outer(current_phase()) {
    current_phase() = n;
  }
  ~Phase() {
    current_phase() = outer;
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    cudaStreamSynchronize(s);
    host_phase(name, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
  }
};

// A sequence of consecutive phases: next() closes the current phase and opens another.
struct PhaseSeq {
  const char* name = nullptr;
  cudaStream_t s;
  std::chrono::steady_clock::time_point t0;
  const char* outer;
  explicit PhaseSeq(cudaStream_t st) : s(st), outer(current_phase()) {}
  void close() {
    current_phase() = outer;
    if (name && g_enabled.load(std::memory_order_relaxed)) {
      cudaStreamSynchronize(s);
      host_phase(name, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    }
    name = nullptr;
  }
  void next(const char* n) {
    close();
    name = n;
    current_phase() = n;
    t0 = std::chrono::steady_clock::now();
  }
  ~PhaseSeq() { close(); }
};

}  // namespace prof
}  // namespace hbs
