// C ABI of the library (include/hbsqp.h): argument checks, handle lifetime, error codes.
#include <chrono>
#include <mutex>
#include <cmath>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "dense_kernels.cuh"
#include "profile.hpp"
#include "qp_kernels.cuh"

namespace hbs {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

bool& gemm_double_float() {
  static thread_local bool df = false;
  return df;
}

bool& gemm_tensor() {
  static thread_local bool tc = false;
  return tc;
}

bool& background_chain() {
  static thread_local bool bg = false;
  return bg;
}

std::mutex& coop_mutex() {
  static std::mutex mu;
  return mu;
}

cudaStream_t& current_stream() {
  static thread_local cudaStream_t s = nullptr;
  return s;
}

namespace {
// Pinned host blocks for read_to_host, kept for the life of the process (never freed:
// cudaFreeHost would synchronize the device).
struct PinnedPool {
  std::mutex mu;
  std::vector<std::pair<void*, size_t>> free;
};
PinnedPool& pinned_pool() {
  static PinnedPool* p = new PinnedPool;
  return *p;
}
}  // namespace

void read_to_host(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return;
  PinnedPool& pool = pinned_pool();
  void* blk = nullptr;
  size_t cap = 0;
  {
    std::lock_guard<std::mutex> lk(pool.mu);
    size_t best = pool.free.size();
    for (size_t i = 0; i < pool.free.size(); ++i)
      if (pool.free[i].second >= bytes && (best == pool.free.size() || pool.free[i].second < pool.free[best].second))
        best = i;
    if (best < pool.free.size()) {
      blk = pool.free[best].first;
      cap = pool.free[best].second;
      pool.free.erase(pool.free.begin() + (std::ptrdiff_t)best);
    }
  }
  if (!blk) {
    cap = 64 * 1024;
    while (cap < bytes) cap *= 2;
    if (cudaMallocHost(&blk, cap) != cudaSuccess) {
      cudaGetLastError();
      blk = nullptr;
    }
  }
  if (!blk) {  // no pinned memory to be had: copy into the caller's memory directly
    HBS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
    HBS_CUDA(cudaStreamSynchronize(s));
    return;
  }
  cudaError_t e = cudaMemcpyAsync(blk, src, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) std::memcpy(dst, blk, bytes);
  {
    std::lock_guard<std::mutex> lk(pool.mu);
    pool.free.push_back({blk, cap});
  }
  cuda_check(e, "read_to_host");
}

// Keep freed memory in the device's default pool (the library frees and reallocates
// work arrays at every level and batch); the pool belongs to this process's context.
void init_memory_pool() {
  static std::once_flag once[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return; }
  std::call_once(once[dev], [dev] {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      // A block freed on one stream is reused by another only once the free has completed:
      // the build's two concurrent chains never wait on each other's kernels through the
      // allocator (with internal dependencies allowed, an allocation on the compression
      // chain's stream could be made to wait for the periodizer's queued launches).
      int no = 0;
      cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    cudaGetLastError();
  });
}

size_t Handle::device_bytes() const {
  size_t b = x.bytes() + y.bytes() + nx.bytes() + ny.bytes() + w.bytes() + Groot.bytes();
  for (const auto& lv : levels)
    b += lv.idx.bytes() + lv.perm.bytes() + lv.T.bytes() + lv.E.bytes() + lv.F.bytes() + lv.G.bytes() +
         lv.Dhat.bytes() + lv.cx.bytes() + lv.cy.bytes() + lv.rad.bytes();
  b += nb_skel.bytes() + Pnb.bytes() + Rm.bytes() + Rp.bytes() + Esamp.bytes() + VT.bytes() + Pdir.bytes() + Zc.bytes() + EZ.bytes() + PE.bytes() + TY.bytes() + TC.bytes() +
       TE.bytes() + Rsel.bytes();
  for (const auto& c : contours)
    b += c.dk.bytes() + c.dwk.bytes() + c.CL.bytes() + c.CR.bytes() + c.SL.bytes() + c.SR.bytes() + c.Zd.bytes();
  return b;
}

template <typename F>
static hbs_status guarded(F&& f) {
  try {
    f();
    return HBS_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return HBS_ERR_OOM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return HBS_ERR_INTERNAL;
  }
}

__global__ void k_kernel_block(DevGeom g, int kind, double shift_x, const int64_t* rows, int64_t nr,
                               const int64_t* cols, int64_t nc, cplx* out) {
  const int64_t tot = nr * nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = rows[e % nr], c = cols[e / nr];
    out[e] = kind == 0 ? a_entry(g, r, c) : a_image_entry(g, r, c, shift_x);
  }
}

// Each node's geometry at both of its unknowns (transmission: out[2p] = out[2p + 1] = in[p]).
__global__ void k_dup2(const double* in, int64_t n, double* out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double v = in[p];
    out[2 * p] = v;
    out[2 * p + 1] = v;
  }
}

// Copy the caller's geometry into device SoA arrays and derive normals and weights; for the
// transmission problem (comps = 2) the arrays are laid out per unknown.
static void load_geometry(Handle& h, const hbs_geometry* geom, cudaStream_t s) {
  const int64_t N = geom->n;
  h.nodes = N;
  h.N = N * h.comps;
  h.d = geom->d;
  DevBuf<double> x(N), y(N), nx(N), ny(N), w(N);
  DevBuf<double> dx(N), dy(N);
  const cudaMemcpyKind kind = geom->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  HBS_CUDA(cudaMemcpyAsync(x.get(), geom->x, N * sizeof(double), kind, s));
  HBS_CUDA(cudaMemcpyAsync(y.get(), geom->y, N * sizeof(double), kind, s));
  HBS_CUDA(cudaMemcpyAsync(dx.get(), geom->dx, N * sizeof(double), kind, s));
  HBS_CUDA(cudaMemcpyAsync(dy.get(), geom->dy, N * sizeof(double), kind, s));
  {
    prof::KScope _ks("k_geom", s);
    k_geom<<<grid_1d(N), 256, 0, s>>>(dx.get(), dy.get(), nx.get(), ny.get(), w.get(), N);
  }
  HBS_LAUNCH_CHECK("k_geom");
  if (h.comps == 1) {
    h.x = std::move(x); h.y = std::move(y); h.nx = std::move(nx); h.ny = std::move(ny); h.w = std::move(w);
  } else {
    DevBuf<double>* src[5] = {&x, &y, &nx, &ny, &w};
    DevBuf<double>* dst[5] = {&h.x, &h.y, &h.nx, &h.ny, &h.w};
    for (int a = 0; a < 5; ++a) {
      dst[a]->alloc(2 * N);
      k_dup2<<<grid_1d(N), 256, 0, s>>>(src[a]->get(), N, dst[a]->get());
    }
    HBS_LAUNCH_CHECK("k_dup2");
  }
  h.hx = h.x.download(s);
  h.hy = h.y.download(s);
}

static DevGeom geom_view(const hbs_geometry* geom, double omega, DevBuf<double>& nx, DevBuf<double>& ny,
                         DevBuf<double>& w, cudaStream_t s) {
  const int64_t N = geom->n;
  nx.alloc(N); ny.alloc(N); w.alloc(N);
  {
    prof::KScope _ks("k_geom", s);
    k_geom<<<grid_1d(N), 256, 0, s>>>(geom->dx, geom->dy, nx.get(), ny.get(), w.get(), N);
  }
  HBS_LAUNCH_CHECK("k_geom");
  DevGeom g;
  g.x = geom->x; g.y = geom->y; g.nx = nx.get(); g.ny = ny.get(); g.w = w.get(); g.n = N; g.omega = omega;
  g.df = false;
  g.comps = 1;
  g.omega_in = 0.0;
  return g;
}

}  // namespace hbs

using namespace hbs;

extern "C" {

void hbs_default_options(hbs_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->leaf_size = 64;
  o->n_proxy_min = 64;
  o->proxy_rho = 1.5;
  o->precision = HBS_PRECISION_FP64;
}

namespace {

hbs_status check_build_args(const hbs_geometry* geom, double omega, double tol) {
  if (!geom || !geom->x || !geom->y || !geom->dx || !geom->dy) {
    set_last_error("geometry arrays are NULL");
    return HBS_ERR_INVALID_ARG;
  }
  if (geom->n < 64 || !(geom->d > 0) || !(omega > 0) || !(tol > 0 && tol < 1)) {
    set_last_error("need n >= 64, d > 0, omega > 0, 0 < tol < 1");
    return HBS_ERR_INVALID_ARG;
  }
  return HBS_OK;
}

// Options, geometry and the wall check of one solver (before its tree is built).
void prepare_handle(Handle& h, const hbs_geometry* geom, double omega, double tol, const hbs_options* opts,
                    cudaStream_t s) {
  hbs_default_options(&h.opts);
  if (opts) h.opts = *opts;
  if (h.opts.leaf_size < 8) h.opts.leaf_size = 64;
  if (h.opts.n_proxy_min < 8) h.opts.n_proxy_min = 64;
  if (!(h.opts.proxy_rho > 1.0)) h.opts.proxy_rho = 1.5;
  if (h.opts.precision != HBS_PRECISION_FP64 && h.opts.precision != HBS_PRECISION_DOUBLE_FLOAT &&
      h.opts.precision != HBS_PRECISION_TENSOR)
    throw Error(HBS_ERR_INVALID_ARG, "unsupported precision mode");
  if (!(h.opts.index >= 0.0) || !std::isfinite(h.opts.index))
    throw Error(HBS_ERR_INVALID_ARG, "refractive index must be 0 (sound-soft) or positive");
  h.comps = h.opts.index > 0.0 ? 2 : 1;
  h.index = h.opts.index;
  h.omega = omega;
  h.tol = tol;
  load_geometry(h, geom, s);
  for (int64_t i = 0; i < h.N; ++i)
    if (!(std::fabs(h.hx[i]) < 0.5 * h.d)) throw Error(HBS_ERR_INVALID_ARG, "obstacle touches a unit-cell wall");
}

}  // namespace

hbs_status hbs_build(const hbs_geometry* geom, double omega, double tol, const hbs_options* opts, void* stream,
                     hbs_handle** out) {
  if (!out) { set_last_error("out is NULL"); return HBS_ERR_INVALID_ARG; }
  *out = nullptr;
  if (hbs_status st = check_build_args(geom, omega, tol)) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScope scope(s);
  hbs_handle* hh = new (std::nothrow) hbs_handle();
  if (!hh) { set_last_error("host allocation failed"); return HBS_ERR_OOM; }
  hbs_status st = guarded([&] {
    Handle& h = hh->h;
    auto t0 = std::chrono::steady_clock::now();
    prepare_handle(h, geom, omega, tol, opts, s);
    GemmModeScope gm(h.opts.precision);
    build_periodizer(h, s, /*with_hbs=*/true);  // runs the HBS compression alongside
    HBS_CUDA(cudaStreamSynchronize(s));
    h.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  });
  if (st != HBS_OK) {
    delete hh;
    return st;
  }
  *out = hh;
  return HBS_OK;
}

hbs_status hbs_build_batch(const hbs_geometry* geoms, const double* omegas, int64_t count, double tol,
                           const hbs_options* opts, void* stream, hbs_handle** out) {
  if (!out || !geoms || !omegas || count <= 0) {
    set_last_error("bad arguments to hbs_build_batch");
    return HBS_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < count; ++i) out[i] = nullptr;
  for (int64_t i = 0; i < count; ++i)
    if (hbs_status st = check_build_args(geoms + i, omegas[i], tol)) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScope scope(s);
  std::vector<hbs_handle*> hh(count, nullptr);
  for (int64_t i = 0; i < count; ++i) {
    hh[i] = new (std::nothrow) hbs_handle();
    if (!hh[i]) {
      for (auto* p : hh) delete p;
      set_last_error("host allocation failed");
      return HBS_ERR_OOM;
    }
  }
  hbs_status st = guarded([&] {
    auto t0 = std::chrono::steady_clock::now();
    std::vector<Handle*> hs(count);
    for (int64_t i = 0; i < count; ++i) {
      hs[i] = &hh[i]->h;
      prepare_handle(*hs[i], geoms + i, omegas[i], tol, opts, s);
    }
    GemmModeScope gm(hs[0]->opts.precision);
    {
      prof::Phase ph("build:hbs_compress_invert", s);
      build_hbs_multi(hs, s);
    }
    for (Handle* h : hs) build_periodizer(*h, s);
    HBS_CUDA(cudaStreamSynchronize(s));
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (Handle* h : hs) h->build_seconds = sec;
  });
  if (st != HBS_OK) {
    for (auto* p : hh) delete p;
    return st;
  }
  for (int64_t i = 0; i < count; ++i) out[i] = hh[i];
  return HBS_OK;
}

static hbs_status solve_common(hbs_handle* h, const double* theta, int64_t n_theta, void* stream, hbs_result** out,
                               bool plain) {
  if (!h || !out || (n_theta > 0 && !theta) || n_theta < 0) {
    set_last_error("bad arguments to hbs_solve");
    return HBS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  hbs_result* r = new (std::nothrow) hbs_result();
  if (!r) { set_last_error("host allocation failed"); return HBS_ERR_OOM; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScope scope(s);
  hbs_status st = guarded([&] {
    GemmModeScope gm(plain ? HBS_PRECISION_FP64 : h->h.opts.precision);
    solve_angles(h->h, theta, n_theta, plain, r->r, s);
    HBS_CUDA(cudaStreamSynchronize(s));
  });
  if (st != HBS_OK) { delete r; return st; }
  *out = r;
  if (r->r.illcond) {
    set_last_error("a Schur system was singular to working precision");
    return HBS_WARN_ILLCOND;
  }
  return HBS_OK;
}

hbs_status hbs_solve(hbs_handle* h, const double* theta, int64_t n_theta, void* stream, hbs_result** out) {
  return solve_common(h, theta, n_theta, stream, out, false);
}

hbs_status hbs_solve_plain(hbs_handle* h, const double* theta, int64_t n_theta, void* stream, hbs_result** out) {
  return solve_common(h, theta, n_theta, stream, out, true);
}

hbs_status hbs_solve_proxy(hbs_handle* h, const double* theta, int64_t n_theta, void* stream, hbs_result** out) {
  if (!h || !out || (n_theta > 0 && !theta) || n_theta < 0) {
    set_last_error("bad arguments to hbs_solve_proxy");
    return HBS_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < n_theta; ++i)
    if (!(theta[i] < 0.0 && theta[i] > -M_PI)) {
      set_last_error("hbs_solve_proxy: incident angles must lie in (-pi, 0)");
      return HBS_ERR_INVALID_ARG;
    }
  *out = nullptr;
  hbs_result* r = new (std::nothrow) hbs_result();
  if (!r) { set_last_error("host allocation failed"); return HBS_ERR_OOM; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScope scope(s);
  hbs_status st = guarded([&] {
    GemmModeScope gm(HBS_PRECISION_FP64);
    solve_angles_proxy(h->h, theta, n_theta, r->r, s);
    HBS_CUDA(cudaStreamSynchronize(s));
  });
  if (st != HBS_OK) { delete r; return st; }
  *out = r;
  return HBS_OK;
}

hbs_status hbs_bragg_amplitudes(const hbs_result* r, int64_t i, int* n_min, int* n_max, double* c, double* d,
                                double* flux_err) {
  if (!r || i < 0 || i >= (int64_t)r->r.angles.size()) {
    set_last_error("bad result or angle index");
    return HBS_ERR_INVALID_ARG;
  }
  const AngleResult& a = r->r.angles[i];
  if (n_min) *n_min = a.n_min;
  if (n_max) *n_max = a.n_max;
  if (flux_err) *flux_err = a.flux_err;
  for (size_t o = 0; o < a.c.size(); ++o) {
    if (c) { c[2 * o] = a.c[o].real(); c[2 * o + 1] = a.c[o].imag(); }
    if (d) { d[2 * o] = a.d[o].real(); d[2 * o + 1] = a.d[o].imag(); }
  }
  return HBS_OK;
}

hbs_status hbs_result_angle_info(const hbs_result* r, int64_t i, int* n_wood, double* t0) {
  if (!r || i < 0 || i >= (int64_t)r->r.angles.size()) {
    set_last_error("bad result or angle index");
    return HBS_ERR_INVALID_ARG;
  }
  if (n_wood) *n_wood = r->r.angles[i].n_wood;
  if (t0) *t0 = r->r.angles[i].t0;
  return HBS_OK;
}

hbs_status hbs_info(const hbs_handle* hh, hbs_info_t* info) {
  if (!hh || !info) { set_last_error("NULL argument"); return HBS_ERR_INVALID_ARG; }
  const Handle& h = hh->h;
  info->n = h.nodes;
  info->unknowns = h.N;
  info->index = h.index;
  info->levels = h.L;
  info->max_rank = h.max_rank;
  info->nb_rank = h.nb_rank;
  info->m = h.M;
  info->n_contours = (int)h.contours.size();
  info->device_bytes = h.device_bytes();
  info->build_seconds = h.build_seconds;
  info->factor_bytes = h.factor_bytes;
  info->apply_flops_per_rhs = h.apply_flops;
  info->contour_h = h.ch;
  info->contour_c = h.cc;
  info->contour_w = h.cw;
  info->wood_t0 = h.contours.size() > 1 ? h.contours[1].t0 : 0.0;
  info->n_bragg_samples = h.S;
  info->y0 = h.y0;
  info->nb_radius = h.nb_R;
  info->nb_proxies = h.nb_np;
  info->pid_col_rank = h.rB;
  info->pid_row_rank = h.rC + h.rE;
  info->pid_residual = h.pid_residual;
  info->nb_residual = h.nb_residual;
  return HBS_OK;
}

hbs_status hbs_apply_inverse(const hbs_handle* hh, const void* b, void* x, int64_t nrhs, void* stream) {
  if (!hh || !b || !x || nrhs < 0) { set_last_error("bad arguments to hbs_apply_inverse"); return HBS_ERR_INVALID_ARG; }
  if (b == x) { set_last_error("b and x must not alias"); return HBS_ERR_INVALID_ARG; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScope scope(s);
  return guarded([&] {
    GemmModeScope gm(hh->h.opts.precision);
    hh->h.apply_inverse(static_cast<const cplx*>(b), static_cast<cplx*>(x), nrhs, s);
    HBS_CUDA(cudaStreamSynchronize(s));
  });
}

hbs_status hbs_kernel_block(const hbs_geometry* geom, double omega, int kind, double shift_x, const int64_t* rows,
                            int64_t nr, const int64_t* cols, int64_t nc, void* out, void* stream) {
  if (!geom || !geom->on_device || !rows || !cols || !out || nr < 0 || nc < 0 || (kind != 0 && kind != 1) ||
      geom->n < 13) {
    set_last_error("bad arguments to hbs_kernel_block (geometry must be on the device)");
    return HBS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScope scope(s);
  return guarded([&] {
    DevBuf<double> nx, ny, w;
    DevGeom g = geom_view(geom, omega, nx, ny, w, s);
    if (nr * nc > 0) {
      {
        prof::KScope _ks("k_kernel_block", s);
        k_kernel_block<<<grid_1d(nr * nc), 256, 0, s>>>(g, kind, shift_x, rows, nr, cols, nc, static_cast<cplx*>(out));
      }
      HBS_LAUNCH_CHECK("k_kernel_block");
    }
    HBS_CUDA(cudaStreamSynchronize(s));
  });
}

hbs_status hbs_kernel_block_transmission(const hbs_geometry* geom, double omega, double index, int kind,
                                         double shift_x, const int64_t* rows, int64_t nr, const int64_t* cols,
                                         int64_t nc, void* out, void* stream) {
  if (!geom || !geom->on_device || !rows || !cols || !out || nr < 0 || nc < 0 || (kind != 0 && kind != 1) ||
      geom->n < 13 || !(index > 0.0) || !std::isfinite(index)) {
    set_last_error("bad arguments to hbs_kernel_block_transmission (geometry on the device, index > 0)");
    return HBS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScope scope(s);
  return guarded([&] {
    const int64_t N = geom->n;
    DevBuf<double> nx, ny, w;
    DevGeom g1 = geom_view(geom, omega, nx, ny, w, s);
    DevBuf<double> arr[5];
    const double* src[5] = {g1.x, g1.y, g1.nx, g1.ny, g1.w};
    for (int a = 0; a < 5; ++a) {
      arr[a].alloc(2 * N);
      k_dup2<<<grid_1d(N), 256, 0, s>>>(src[a], N, arr[a].get());
    }
    HBS_LAUNCH_CHECK("k_dup2");
    DevGeom g = g1;
    g.x = arr[0].get(); g.y = arr[1].get(); g.nx = arr[2].get(); g.ny = arr[3].get(); g.w = arr[4].get();
    g.n = 2 * N;
    g.comps = 2;
    g.omega_in = index * omega;
    if (nr * nc > 0) {
      {
        prof::KScope _ks("k_kernel_block", s);
        k_kernel_block<<<grid_1d(nr * nc), 256, 0, s>>>(g, kind, shift_x, rows, nr, cols, nc, static_cast<cplx*>(out));
      }
      HBS_LAUNCH_CHECK("k_kernel_block");
    }
    HBS_CUDA(cudaStreamSynchronize(s));
  });
}

hbs_status hbs_zgemm(int64_t m, int64_t n, int64_t k, const double* alpha, const void* a, int64_t lda, int trans_a,
                     const void* b, int64_t ldb, const double* beta, void* c, int64_t ldc, int precision,
                     void* stream) {
  const bool sizes_ok = m >= 0 && n >= 0 && k >= 0 && m <= INT32_MAX && n <= INT32_MAX && k <= INT32_MAX;
  if (!sizes_ok || !alpha || !beta || (precision < HBS_PRECISION_FP64 || precision > HBS_PRECISION_TENSOR) ||
      ldc < std::max<int64_t>(1, m) || ldb < std::max<int64_t>(1, k) ||
      lda < std::max<int64_t>(1, trans_a ? k : m) || lda > INT32_MAX || ldb > INT32_MAX || ldc > INT32_MAX ||
      (m > 0 && n > 0 && (!c || (k > 0 && (!a || !b))))) {
    set_last_error("bad arguments to hbs_zgemm");
    return HBS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScope scope(s);
  return guarded([&] {
    if (m == 0 || n == 0) return;
    GemmModeScope gm(precision);
    GemmJob j{};
    j.A = static_cast<const cplx*>(a);
    j.B = static_cast<const cplx*>(b);
    j.C = static_cast<cplx*>(c);
    j.m = (int)m;
    j.n = (int)n;
    j.k = (int)k;
    j.lda = (int)lda;
    j.ldb = (int)ldb;
    j.ldc = (int)ldc;
    j.alpha = cmk(alpha[0], alpha[1]);
    j.beta = cmk(beta[0], beta[1]);
    j.transA = trans_a ? 1 : 0;
    std::vector<GemmJob> jobs{j};
    run_gemms(jobs, s);
    HBS_CUDA(cudaStreamSynchronize(s));
  });
}

hbs_status hbs_row_id(void* mt, int64_t m, int64_t n, double tol, int* rank, int* perm, void* t, void* stream) {
  if (!mt || !rank || !perm || !t || m <= 0 || n <= 0 || !(tol > 0)) {
    set_last_error("bad arguments to hbs_row_id");
    return HBS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScope scope(s);
  return guarded([&] {
    if (n <= 4096) {
      std::vector<CpqrJob> jobs(1);
      jobs[0] = {static_cast<cplx*>(mt), static_cast<cplx*>(t), perm, (int)m, (int)n, 0};
      auto r = batched_id(jobs, tol, s);
      *rank = r[0];
    } else {
      *rank = big_row_id(static_cast<cplx*>(mt), m, n, tol, perm, static_cast<cplx*>(t),
                         (int)std::min<int64_t>(m, n), s);
    }
    HBS_CUDA(cudaStreamSynchronize(s));
  });
}

hbs_status hbs_batched_inverse(void* a, int64_t n, int64_t count, int precision, void* stream) {
  if (!a || n < 1 || n > 4096 || count < 1 || count > (1 << 20) || precision < HBS_PRECISION_FP64 ||
      precision > HBS_PRECISION_TENSOR) {
    set_last_error("bad arguments to hbs_batched_inverse");
    return HBS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScope scope(s);
  GemmModeScope mode(precision);
  return guarded([&] {
    std::vector<InvJob> jobs((size_t)count);
    for (int64_t i = 0; i < count; ++i) jobs[i] = {static_cast<cplx*>(a) + i * n * n, nullptr, (int)n, (int)i};
    batched_inverse(jobs, s, "hbs_batched_inverse");
    HBS_CUDA(cudaStreamSynchronize(s));
  });
}

hbs_status hbs_save(const hbs_handle* h, const char* path, void* stream) {
  if (!h || !path) {
    set_last_error("bad arguments to hbs_save");
    return HBS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScope scope(s);
  return guarded([&] { save_handle(const_cast<hbs_handle*>(h)->h, path, s); });
}

hbs_status hbs_load(const char* path, void* stream, hbs_handle** out) {
  if (!out) { set_last_error("out is NULL"); return HBS_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!path) { set_last_error("path is NULL"); return HBS_ERR_INVALID_ARG; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScope scope(s);
  hbs_handle* hh = new (std::nothrow) hbs_handle();
  if (!hh) { set_last_error("host allocation failed"); return HBS_ERR_OOM; }
  hbs_status st = guarded([&] { load_handle(hh->h, path, s); });
  if (st != HBS_OK) {
    delete hh;
    return st;
  }
  *out = hh;
  return HBS_OK;
}

void hbs_free(hbs_handle* h) {
  if (!h) return;
  // the handle's buffers are freed in stream order on the legacy stream; finish all work first
  cudaDeviceSynchronize();
  StreamScope scope(nullptr);
  delete h;
  cudaDeviceSynchronize();
  cudaGetLastError();
}
void hbs_result_free(hbs_result* r) { delete r; }
const char* hbs_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
