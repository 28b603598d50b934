// Device buffers, status codes and error plumbing shared by the library's host code.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "../../include/hbsqp.h"

namespace hbs {

struct Error : public std::runtime_error {
  hbs_status code;
  Error(hbs_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

inline void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(e == cudaErrorMemoryAllocation ? HBS_ERR_OOM : HBS_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  }
}

#define HBS_CUDA(call) ::hbs::cuda_check((call), #call)
#define HBS_LAUNCH_CHECK(name) ::hbs::cuda_check(cudaGetLastError(), name)

cudaStream_t& current_stream();

// Fault injection for tests of the error paths (hbs_fault_inject): true when the caller's
// device allocation is the one chosen to fail; the largest rank an ID may reach (0 = none).
bool injected_alloc_failure();

// Raise a kernel's limit on dynamic shared memory to at least `bytes` (cudaFuncSetAttribute)
// on the current device.  The limit only ever grows, under a lock: two host threads that
// launch the same kernel with different sizes (the build's two streams) cannot lower it
// between another's occupancy query and its launch.  Returns the runtime's status.
inline cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[{dev, fn}];
  if (bytes <= 48 * 1024 || bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}
int injected_rank_cap();

// Copies `bytes` of device memory at `src` to host memory at `dst` once the stream reaches
// the copy, and returns then.  The copy lands in a pinned staging block (a process-wide pool,
// reused) and is then copied out: a device-to-host copy into pageable memory would hold the
// runtime's pageable-copy path until the stream got there, and a second host thread's
// uploads (the build runs two) would stall behind it meanwhile.
void read_to_host(void* dst, const void* src, size_t bytes, cudaStream_t s);

// Owning device allocation (stream-ordered cudaMallocAsync / cudaFreeAsync on the
// library's current stream).
template <typename T>
class DevBuf {
 public:
  DevBuf() = default;
  explicit DevBuf(size_t n) { alloc(n); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p_(o.p_), n_(o.n_) { o.p_ = nullptr; o.n_ = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p_ = o.p_; n_ = o.n_; o.p_ = nullptr; o.n_ = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t n) {
    release();
    if (n == 0) return;
    void* p = nullptr;
    if (injected_alloc_failure())
      throw Error(HBS_ERR_OOM, "device allocation failed (injected by hbs_fault_inject)");
    HBS_CUDA(cudaMallocAsync(&p, n * sizeof(T), current_stream()));
    p_ = static_cast<T*>(p);
    n_ = n;
  }
  void release() {
    if (p_) cudaFreeAsync(p_, current_stream());
    p_ = nullptr;
    n_ = 0;
  }
  T* get() const { return p_; }
  size_t size() const { return n_; }
  size_t bytes() const { return n_ * sizeof(T); }
  void upload(const std::vector<T>& h, cudaStream_t s) {
    if (h.size() > n_) alloc(h.size());
    if (!h.empty())
      HBS_CUDA(cudaMemcpyAsync(p_, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  std::vector<T> download(cudaStream_t s, size_t count = SIZE_MAX) const {
    size_t c = count == SIZE_MAX ? n_ : count;
    std::vector<T> h(c);
    if (c) read_to_host(h.data(), p_, c * sizeof(T), s);
    return h;
  }

 private:
  T* p_ = nullptr;
  size_t n_ = 0;
};

void set_last_error(const std::string& msg);

// Stream on which the library allocates and frees device memory.  Every C entry point
// that works on a stream installs it for its duration (StreamScope); allocations are
// stream ordered (cudaMallocAsync / cudaFreeAsync from the device's memory pool), so
// freeing a buffer does not synchronize the device and memory is reused in stream order.
cudaStream_t& current_stream();
void init_memory_pool();

// Arithmetic of the library's batched GEMMs on this thread: FP64 (false) or double-float
// (true), set for the duration of a call from the handle's precision option.
bool& gemm_double_float();

// Held from the launch of a cooperative (grid-barrier) kernel until the host has seen it
// finish: at most one such kernel is in flight on the device, whatever the number of
// threads and streams using the library.
std::mutex& coop_mutex();
// Large products on the tensor cores (digit-plane splitting) on this thread.
bool& gemm_tensor();
// True on the thread that builds the periodizer while another thread runs the compression
// chain (the build's critical path) on a higher-priority stream: this thread's persistent
// QRs take one CTA per SM instead of two and leave half of every SM to the compression.
bool& background_chain();

// Sets the thread's arithmetic modes from an HBS_PRECISION_* value for a call's duration.
struct GemmModeScope {
  bool prev, prev_tc;
  explicit GemmModeScope(int precision) : prev(gemm_double_float()), prev_tc(gemm_tensor()) {
    gemm_double_float() = precision == HBS_PRECISION_DOUBLE_FLOAT || precision == HBS_PRECISION_TENSOR;
    gemm_tensor() = precision == HBS_PRECISION_TENSOR;
  }
  ~GemmModeScope() {
    gemm_double_float() = prev;
    gemm_tensor() = prev_tc;
  }
};

struct StreamScope {
  cudaStream_t prev;
  explicit StreamScope(cudaStream_t s) : prev(current_stream()) {
    init_memory_pool();
    current_stream() = s;
  }
  ~StreamScope() { current_stream() = prev; }
};

}  // namespace hbs
