// Launch accounting and per-kernel CUDA-event timing (see profile.hpp).  With the
// environment variable HBS_PROFILE_TIMELINE naming a file, every profiled launch is also
// written there as one CSV line (kernel, phase, stream, device start and duration in ms, the
// start measured from an event recorded when profiling was switched on, and the host time
// at which the launch was issued, from the same moment on the host clock).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "devbuf.hpp"
#include "profile.hpp"

namespace hbs {
namespace prof {

std::atomic<int64_t> g_launches{0};
std::atomic<int> g_enabled{0};

namespace {
struct Pending {
  std::string name;
  const char* phase;
  cudaStream_t s;
  cudaEvent_t a, b;
  double flops, bytes;
  std::chrono::steady_clock::time_point issued;
};
struct Stat {
  int64_t launches = 0;
  double ms = 0.0, flops = 0.0, bytes = 0.0;
};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::map<std::string, Stat> g_stats;
std::vector<cudaEvent_t> g_free;
FILE* g_timeline = nullptr;
cudaEvent_t g_origin = nullptr;
std::chrono::steady_clock::time_point g_origin_host;

void drain_locked() {
  for (auto& p : g_pending) {
    cudaEventSynchronize(p.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    Stat& st = g_stats[p.name];
    st.launches += 1;
    st.ms += ms;
    st.flops += p.flops;
    st.bytes += p.bytes;
    if (p.phase) {
      // the same launch charged to its phase: "in:<phase>:<kernel>", time and launches only
      Stat& sp = g_stats[std::string("in:") + p.phase + ":" + p.name];
      sp.launches += 1;
      sp.ms += ms;
    }
    if (g_timeline && g_origin) {
      float t0 = 0.f;
      if (cudaEventElapsedTime(&t0, g_origin, p.a) == cudaSuccess)
        std::fprintf(g_timeline, "%s,%s,%p,%.4f,%.4f,%.4f\n", p.name.c_str(), p.phase ? p.phase : "", (void*)p.s, t0,
                     ms, 1e3 * std::chrono::duration<double>(p.issued - g_origin_host).count());
      else
        cudaGetLastError();
    }
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.clear();
}
}  // namespace

cudaEvent_t new_event() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void record(const char* name, const char* phase, cudaStream_t s, cudaEvent_t a, cudaEvent_t b, double flops,
            double bytes, std::chrono::steady_clock::time_point issued) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_pending.push_back({name, phase, s, a, b, flops, bytes, issued});
  if (g_pending.size() > 4096) drain_locked();
}

void add_work(const char* name, double flops, double bytes) {
  if (!g_enabled.load()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Stat& st = g_stats[name];
  st.flops += flops;
  st.bytes += bytes;
}

void host_phase(const char* name, double seconds) {
  if (!g_enabled.load()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Stat& st = g_stats[std::string("phase:") + name];
  st.ms += 1e3 * seconds;
}

}  // namespace prof
}  // namespace hbs

using namespace hbs::prof;

extern "C" {

void hbs_profile_enable(int on) {
  if (on) {
    std::lock_guard<std::mutex> lk(g_mu);
    const char* path = std::getenv("HBS_PROFILE_TIMELINE");
    if (path && *path && !g_timeline) {
      g_timeline = std::fopen(path, "w");
      if (g_timeline) std::fprintf(g_timeline, "kernel,phase,stream,start_ms,ms,issued_ms\n");
    }
    if (g_timeline) {
      if (!g_origin) cudaEventCreate(&g_origin);
      cudaEventRecord(g_origin, 0);
      g_origin_host = std::chrono::steady_clock::now();
    }
  }
  g_enabled.store(on ? 1 : 0);
}

void hbs_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  g_stats.clear();
}

int hbs_profile_get(hbs_kernel_stat* out, int max) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  if (g_timeline) std::fflush(g_timeline);
  int i = 0;
  for (auto& kv : g_stats) {
    if (out && i < max) {
      std::memset(&out[i], 0, sizeof(hbs_kernel_stat));
      std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
      out[i].launches = kv.second.launches;
      out[i].ms = kv.second.ms;
      out[i].flops = kv.second.flops;
      out[i].bytes = kv.second.bytes;
    }
    ++i;
  }
  return i;
}

int64_t hbs_launch_count(void) { return g_launches.load(); }

}  // extern "C"
