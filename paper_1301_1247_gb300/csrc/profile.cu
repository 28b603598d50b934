// Launch accounting and per-kernel CUDA-event timing (see profile.hpp).
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
  cudaEvent_t a, b;
  double flops, bytes;
};
struct Stat {
  int64_t launches = 0;
  double ms = 0.0, flops = 0.0, bytes = 0.0;
};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::map<std::string, Stat> g_stats;
std::vector<cudaEvent_t> g_free;

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

void record(const char* name, cudaStream_t, cudaEvent_t a, cudaEvent_t b, double flops, double bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_pending.push_back({name, a, b, flops, bytes});
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

void hbs_profile_enable(int on) { g_enabled.store(on ? 1 : 0); }

void hbs_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  g_stats.clear();
}

int hbs_profile_get(hbs_kernel_stat* out, int max) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
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
