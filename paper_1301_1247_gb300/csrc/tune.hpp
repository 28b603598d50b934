// Launch-shape autotuner for the batched kernels.
//
// A tuned call site names its kernel family and shape class (a key such as
// "bgj/n512/b4") and the number of launch variants it can run.  With tuning on
// (HBS_AUTOTUNE=1 in the environment), the first calls for a key run each variant once,
// timed with CUDA events on the launching stream, and later calls run the fastest.  The
// measured choices are read from and written to the file named by HBS_TUNE_FILE (one
// "key variant milliseconds" line per key), so a later process starts from them.  With
// tuning off, a key takes its stored choice if the file has one, else the call site's
// default.  Variants of one call site compute the same result up to rounding.
#pragma once

#include <cuda_runtime.h>

#include <string>

namespace hbs {
namespace tune {

// The variant to run now for `key` (0 <= v < count); `fallback` when nothing is known.
int choose(const std::string& key, int count, int fallback);
// True while `key` still has unmeasured variants (the call should then be timed).
bool exploring(const std::string& key, int count);
// The measured time of `variant` for `key`.
void record(const std::string& key, int variant, int count, float ms);

// Times the enclosed launches on stream s when the key is being explored.
struct Timed {
  std::string key;
  int variant, count;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  Timed(std::string k, int v, int c, cudaStream_t st);
  ~Timed();
};

}  // namespace tune
}  // namespace hbs
