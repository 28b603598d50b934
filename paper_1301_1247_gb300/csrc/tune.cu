// Launch-shape autotuner (tune.hpp): per-key measurements, the choice of the fastest
// variant, and the optional file that keeps the choices between processes.
#include "tune.hpp"

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

namespace hbs {
namespace tune {
namespace {

struct Entry {
  std::vector<float> ms;  // per variant, < 0: not measured
  int best = -1;          // chosen variant once all are measured (or read from the file)
};

std::mutex g_mu;
std::map<std::string, Entry> g_tab;
bool g_loaded = false;

bool enabled() {
  const char* v = std::getenv("HBS_AUTOTUNE");
  return v && v[0] && std::strcmp(v, "0") != 0;
}

const char* tune_file() {
  const char* f = std::getenv("HBS_TUNE_FILE");
  return (f && f[0]) ? f : nullptr;
}

void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const char* f = tune_file();
  if (!f) return;
  FILE* fp = std::fopen(f, "r");
  if (!fp) return;
  char key[256];
  int v = 0;
  float ms = 0.f;
  while (std::fscanf(fp, "%255s %d %f", key, &v, &ms) == 3)
    if (v >= 0) g_tab[key].best = v;
  std::fclose(fp);
}

void save_locked() {
  const char* f = tune_file();
  if (!f) return;
  FILE* fp = std::fopen(f, "w");
  if (!fp) return;
  for (const auto& kv : g_tab) {
    if (kv.second.best < 0) continue;
    const int b = kv.second.best;
    const float ms = b < (int)kv.second.ms.size() ? kv.second.ms[b] : -1.f;
    std::fprintf(fp, "%s %d %.6f\n", kv.first.c_str(), b, ms);
  }
  std::fclose(fp);
}

Entry& entry_locked(const std::string& key, int count) {
  Entry& e = g_tab[key];
  if ((int)e.ms.size() < count) e.ms.resize(count, -1.f);
  return e;
}

}  // namespace

bool exploring(const std::string& key, int count) {
  if (!enabled() || count < 2) return false;
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  const Entry& e = entry_locked(key, count);
  for (int v = 0; v < count; ++v)
    if (e.ms[v] < 0.f) return true;
  return false;
}

int choose(const std::string& key, int count, int fallback) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  Entry& e = entry_locked(key, count);
  if (enabled() && count > 1)
    for (int v = 0; v < count; ++v)
      if (e.ms[v] < 0.f) return v;  // explore the next unmeasured variant
  if (e.best >= 0 && e.best < count) return e.best;
  return fallback;
}

void record(const std::string& key, int variant, int count, float ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  Entry& e = entry_locked(key, count);
  if (variant < 0 || variant >= count) return;
  e.ms[variant] = ms;
  int best = -1;
  for (int v = 0; v < count; ++v) {
    if (e.ms[v] < 0.f) return;  // still exploring
    if (best < 0 || e.ms[v] < e.ms[best]) best = v;
  }
  e.best = best;
  save_locked();
}

Timed::Timed(std::string k, int v, int c, cudaStream_t st) : key(std::move(k)), variant(v), count(c), s(st) {
  if (!exploring(key, count)) return;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    a = b = nullptr;
    return;
  }
  cudaEventRecord(a, s);
}

Timed::~Timed() {
  if (!a) return;
  float ms = -1.f;
  if (cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
      cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms >= 0.f)
    record(key, variant, count, ms);
  cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
}

}  // namespace tune
}  // namespace hbs
