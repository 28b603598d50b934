// Allocation-free variant of the multi-CTA interpolative decomposition (hbs_row_id_static).
//
// Some callers cannot allocate device memory while they call into this library: code that
// runs under a fixed, pre-reserved device-memory budget (a serving process that must not
// grow), code that may not block on cudaMalloc / cudaFree (cudaFree synchronizes the whole
// device, which a latency-critical caller cannot afford), and code that sits behind a
// custom allocator it does not control.  hbs_row_id allocates its working arrays on every
// call; this entry point instead keeps them in one file-scope device array of fixed size
// that every GPU loading the library reserves until the process exits.
//
// The working arrays are: squared column norms and their reference values (2 n doubles),
// the per-block partial maxima of the pivot search, and the step state of the QR.  The
// largest supported n is HBS_ROW_ID_STATIC_MAX_N columns.
#include <algorithm>
#include <mutex>
#include <string>

#include "dense_kernels.cuh"
#include "profile.hpp"
#include "qp_kernels.cuh"

namespace hbs {
namespace {

constexpr int64_t kMaxN = HBS_ROW_ID_STATIC_MAX_N;
constexpr int kParts = 296;  // blocks of the pivot search

struct StaticScratch {
  double nrm[kMaxN];
  double nref[kMaxN];
  double pv[kParts];
  int pi[kParts];
  BigQrState st;
};

// One copy per device, resident until the process exits.
static __device__ __align__(256) StaticScratch g_scratch;

// Device address of g_scratch, looked up once per device with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
StaticScratch* g_addr[kMaxDevices] = {nullptr};

StaticScratch* scratch_for_current_device() {
  int dev = 0;
  HBS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw Error(HBS_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      throw Error(HBS_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                    cudaGetErrorString(e));
    }
    g_addr[dev] = static_cast<StaticScratch*>(p);
  }
  return g_addr[dev];
}

int row_id_static(cplx* Mt, int64_t m, int64_t n, double tol, int* perm, cplx* T, cudaStream_t s) {
  StaticScratch* sc = scratch_for_current_device();
  double* nrm = sc->nrm;
  double* nref = sc->nref;
  BigQrState* st = &sc->st;
  // The step state must start at zero; the norm arrays are overwritten by k_bq_norms.
  HBS_CUDA(cudaMemsetAsync(st, 0, sizeof(BigQrState), s));
  {
    prof::KScope _ks("k_bq_norms", s);
    k_bq_norms<<<1184, 256, 0, s>>>(Mt, m, n, nrm, nref, perm);
  }
  HBS_LAUNCH_CHECK("k_bq_norms");
  const int64_t kcap = std::min<int64_t>(m, n);
  BigQrState hs{};
  for (int64_t step = 0; step < kcap; ++step) {
    {
      prof::KScope _ks("k_bq_argmax", s);
      k_bq_argmax<<<kParts, 256, 0, s>>>(nrm, step, n, st, sc->pv, sc->pi);
    }
    {
      prof::KScope _ks("k_bq_pivot", s);
      k_bq_pivot<<<1, 256, 0, s>>>(Mt, m, step, nrm, nref, perm, sc->pv, sc->pi, kParts, st, tol);
    }
    {
      prof::KScope _ks("k_bq_update", s);
      k_bq_update<<<1184, 256, 0, s>>>(Mt, m, n, step, nrm, nref, st);
    }
    if ((step & 15) == 15) {
      HBS_LAUNCH_CHECK("static row id step");
      HBS_CUDA(cudaMemcpyAsync(&hs, st, sizeof(BigQrState), cudaMemcpyDeviceToHost, s));
      HBS_CUDA(cudaStreamSynchronize(s));
      if (hs.done) break;
    }
  }
  HBS_LAUNCH_CHECK("static row id");
  HBS_CUDA(cudaMemcpyAsync(&hs, st, sizeof(BigQrState), cudaMemcpyDeviceToHost, s));
  HBS_CUDA(cudaStreamSynchronize(s));
  const int k = hs.rank;
  if (k > 0 && n > k) {
    prof::KScope _ks("k_bq_tsolve", s);
    k_bq_tsolve<<<1184, 256, 0, s>>>(Mt, m, n, k, T);
  }
  HBS_LAUNCH_CHECK("k_bq_tsolve");
  HBS_CUDA(cudaStreamSynchronize(s));
  return k;
}

}  // namespace
}  // namespace hbs

extern "C" hbs_status hbs_row_id_static(void* mt, int64_t m, int64_t n, double tol, int* rank, int* perm, void* t,
                                        void* stream) {
  if (!mt || !rank || !perm || !t || m <= 0 || n <= 0 || !(tol > 0)) {
    hbs::set_last_error("bad arguments to hbs_row_id_static");
    return HBS_ERR_INVALID_ARG;
  }
  if (n > HBS_ROW_ID_STATIC_MAX_N) {
    hbs::set_last_error("hbs_row_id_static: n exceeds HBS_ROW_ID_STATIC_MAX_N (262144) columns");
    return HBS_ERR_INVALID_ARG;
  }
  try {
    *rank = hbs::row_id_static(static_cast<cplx*>(mt), m, n, tol, perm, static_cast<cplx*>(t),
                               static_cast<cudaStream_t>(stream));
    return HBS_OK;
  } catch (const hbs::Error& e) {
    hbs::set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    hbs::set_last_error(e.what());
    return HBS_ERR_INTERNAL;
  }
}
