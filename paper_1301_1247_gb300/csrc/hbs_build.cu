// HBS compression and inversion of the isolated-obstacle matrix A (Sec. 4) and the
// telescoping apply of its compressed inverse.
//
// Tree: a balanced binary tree over contiguous index ranges; level l has 2^l nodes,
// node j of level l owns the boundary nodes [j N / 2^l, (j+1) N / 2^l).  Leaves are
// at level L with at most `leaf_size` points.
//
// Compression (leaf to root).  For each node tau with index set I_tau (all points of a
// leaf; the union of the children's skeletons above), one joint interpolative
// decomposition (Def. 3.1) of
//     [ A(I_tau, near) | proxy sources -> I_tau | A(near, I_tau)^T | I_tau -> proxy field ]
// picks skeleton rows J_tau and P_tau with A(I_tau, far) ~ P_tau A(J_tau, far) and
// A(far, I_tau) ~ A(far, J_tau) P_tau^T.  "near" are the active points of the other
// nodes of the level inside the proxy circle (radius rho r_tau, concentric with the node);
// everything outside is represented by the proxy points on that circle (the potential
// theory argument of Sec. 3.2 applied per node).  This gives the block-separable form
// of Eq. (yy2) with U = P, V* = P^T and off-diagonal skeleton blocks A(J_sigma, J_tau).
//
// Inversion (Eqs. woodbury, def_muhD..def_muG), per node:
//     D_tau = A(I_tau, I_tau)                          (leaf)
//     D_tau = [[Dhat_a, A(J_a, J_b)], [A(J_b, J_a), Dhat_b]]   (children a, b)
//     Dhat = (P^T D^{-1} P)^{-1},  E = D^{-1} P Dhat,  F* = Dhat P^T D^{-1},
//     G = D^{-1} - D^{-1} P Dhat P^T D^{-1},
// and the root block [[Dhat_a, A(J_a,J_b)], [A(J_b,J_a), Dhat_b]] is inverted densely.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>

#include "dense_kernels.cuh"
#include "profile.hpp"
#include "handle.hpp"
#include "qp_kernels.cuh"
#include "zgemm.cuh"

namespace hbs {

__global__ void k_geom(const double* dx, const double* dy, double* nx, double* ny, double* w, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double sp = sqrt(dx[i] * dx[i] + dy[i] * dy[i]);
  nx[i] = dy[i] / sp;
  ny[i] = -dx[i] / sp;
  w[i] = (2.0 * HBS_PI / (double)n) * sp;
}

__device__ __forceinline__ int64_t node_lo(int64_t j, int l, int64_t N) { return (j * N) >> l; }

// Enclosing circle of the original points of each node on level l: centre of the
// bounding box, radius = largest distance from it.
__global__ void k_node_circles(const double* x, const double* y, int64_t N, int l, double* cx, double* cy,
                               double* rad) {
  __shared__ double red[32];
  const int64_t j = blockIdx.x;
  const int64_t lo = node_lo(j, l, N), hi = node_lo(j + 1, l, N);
  double mnx = 1e300, mxx = -1e300, mny = 1e300, mxy = -1e300;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    mnx = fmin(mnx, x[i]); mxx = fmax(mxx, x[i]);
    mny = fmin(mny, y[i]); mxy = fmax(mxy, y[i]);
  }
  double v[4] = {-mnx, mxx, -mny, mxy};
  for (int q = 0; q < 4; ++q) {
    double t = v[q];
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double r = -1e300;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
      red[31] = r;
    }
    __syncthreads();
    v[q] = red[31];
  }
  const double ccx = 0.5 * (v[1] - v[0]), ccy = 0.5 * (v[3] - v[2]);
  double r2 = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double ddx = x[i] - ccx, ddy = y[i] - ccy;
    r2 = fmax(r2, ddx * ddx + ddy * ddy);
  }
  for (int o = 16; o > 0; o >>= 1) r2 = fmax(r2, __shfl_xor_sync(0xffffffffu, r2, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    cx[j] = ccx;
    cy[j] = ccy;
    rad[j] = sqrt(r);
  }
}

// Near lists: active points of other nodes of the level inside node tau's proxy circle.
// One block per node scans the level's active points in order, so the list order is
// deterministic.  With `out` == nullptr only the count is produced.
__global__ void k_near(const double* x, const double* y, const int64_t* idx, int64_t ntot, const int64_t* off,
                       const int* nn, const double* cx, const double* cy, const double* rad, double rho,
                       int64_t* count, const int64_t* out_off, int64_t* out) {
  __shared__ int wsum[32];
  __shared__ int64_t base;
  const int tau = blockIdx.x;
  const int64_t own_lo = off[tau], own_hi = off[tau] + nn[tau];
  const double R = rho * rad[tau], R2 = R * R, ccx = cx[tau], ccy = cy[tau];
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t p0 = 0; p0 < ntot; p0 += blockDim.x) {
    int64_t p = p0 + threadIdx.x;
    bool f = false;
    int64_t g = 0;
    if (p < ntot && (p < own_lo || p >= own_hi)) {
      g = idx[p];
      double ddx = x[g] - ccx, ddy = y[g] - ccy;
      f = ddx * ddx + ddy * ddy < R2;
    }
    unsigned b = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[warp] = __popc(b);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) before += wsum[w];
      total += wsum[w];
    }
    if (f && out) out[out_off[tau] + base + before + __popc(b & ((1u << lane) - 1u))] = g;
    __syncthreads();
    if (threadIdx.x == 0) base += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) count[tau] = base;
}

struct YJob {
  int64_t mt_off;    // into the Y pool
  int64_t idx_off;   // into level idx
  int64_t near_off;  // into near list
  int n, nn, np;
  double cx, cy, R, wp;
};

// Fill Mt = Y^T (m x n, m = 2 nn + 2 np): columns are the node's points.  Proxy rows: the
// combined layer dG/dn_p - i w G of proxy sources acting on the node (outside -> in; no
// Fourier mode of the disk is missed since H_m' - i H_m never vanishes on the real axis),
// then the node's field at the proxy points (in -> out; the exterior Dirichlet data
// determine a radiating field).
// Entries come in pairs that share one Hankel evaluation: A(near_r, j) and A(j, near_r)
// (rows r and nn + r), and the combined-layer proxy row and the field-at-proxy column of
// proxy p (rows 2nn + p and 2nn + np + p) -- each pair has a single distance |x - y|.
__global__ void k_fill_y(DevGeom g, const YJob* jobs, const int64_t* idx, const int64_t* near, cplx* pool) {
  const YJob jb = jobs[blockIdx.y];
  const int m = 2 * jb.nn + 2 * jb.np;
  const int half = jb.nn + jb.np;
  const int64_t tot = (int64_t)half * jb.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % half), c = (int)(e / half);
    const int64_t gj = idx[jb.idx_off + c];
    cplx* col = pool + jb.mt_off + (int64_t)c * m;
    const double xj = g.x[gj], yj = g.y[gj];
    if (r < jb.nn) {
      const int64_t gi = near[jb.near_off + r];
      cplx v1, v2;
      if (gi == gj) {
        v1 = v2 = cmk(0.5, 0.0);
      } else {
        const double dx = g.x[gi] - xj, dy = g.y[gi] - yj;
        const double rr = sqrt(dx * dx + dy * dy);
        cplx h0, h1;
        hankel01(g.omega * rr, &h0, &h1);
        const double q = 0.25 * g.omega / rr;
        const double kw = kr6_weight(gi, gj, g.n);
        // A(gi, gj): target gi, source gj;  A(gj, gi): target gj, source gi
        v1 = cscale(combined_from(q * (dx * g.nx[gj] + dy * g.ny[gj]), h0, h1, g.omega), kw * g.w[gj]);
        v2 = cscale(combined_from(-q * (dx * g.nx[gi] + dy * g.ny[gi]), h0, h1, g.omega), kw * g.w[gi]);
      }
      col[r] = v1;
      col[jb.nn + r] = v2;
    } else {
      const int p = r - jb.nn;
      const double th = 2.0 * HBS_PI * (double)p / (double)jb.np;
      double sn, cs;
      sincos(th, &sn, &cs);
      const double px = jb.cx + jb.R * cs, py = jb.cy + jb.R * sn;
      const double dx = xj - px, dy = yj - py;
      const double rr = sqrt(dx * dx + dy * dy);
      cplx h0, h1;
      hankel01(g.omega * rr, &h0, &h1);
      const double q = 0.25 * g.omega / rr;
      // combined-layer source at the proxy (normal = radial direction), target node j
      col[2 * jb.nn + p] = cscale(combined_from(q * (dx * cs + dy * sn), h0, h1, g.omega), jb.wp);
      // field at the proxy of the node's source j
      col[2 * jb.nn + jb.np + p] =
          cscale(combined_from(-q * (dx * g.nx[gj] + dy * g.ny[gj]), h0, h1, g.omega), g.w[gj]);
    }
  }
}

struct DJob {
  int64_t d_off;      // into D pool (n x n)
  int64_t idx_off;    // level idx offset of the node
  int n, k0;          // node size; first child's skeleton size (0 for leaves)
  int leaf;
  const cplx* dh0;    // children's Dhat (k0 x k0, k1 x k1)
  const cplx* dh1;
};

__global__ void k_fill_d(DevGeom g, const DJob* jobs, const int64_t* idx, cplx* pool) {
  const DJob jb = jobs[blockIdx.y];
  const int n = jb.n;
  const int64_t tot = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % n), c = (int)(e / n);
    cplx v;
    if (jb.leaf) {
      v = a_entry(g, idx[jb.idx_off + r], idx[jb.idx_off + c]);
    } else {
      const int k0 = jb.k0, k1 = n - k0;
      const bool r0 = r < k0, c0 = c < k0;
      if (r0 && c0) v = jb.dh0[(int64_t)c * k0 + r];
      else if (!r0 && !c0) v = jb.dh1[(int64_t)(c - k0) * k1 + (r - k0)];
      else v = a_entry(g, idx[jb.idx_off + r], idx[jb.idx_off + c]);
    }
    pool[jb.d_off + e] = v;
  }
}

struct PJob {
  const cplx* in;   // input matrix
  cplx* out;
  const int* perm;  // n entries
  const cplx* T;    // k x (n - k), ld = k
  int n, k;
  int other;        // the other dimension (rows of In for right-P, columns for left-P^T)
  int ld_in, ld_out;
};

// out = In * P  (In: other x n, out: other x k):  out[:, i] = In[:, perm[i]] + sum_j T[i, j] In[:, perm[k + j]]
__global__ void k_right_p(const PJob* jobs) {
  const PJob jb = jobs[blockIdx.y];
  const int64_t tot = (int64_t)jb.other * jb.k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % jb.other), i = (int)(e / jb.other);
    cplx acc = jb.in[(int64_t)jb.perm[i] * jb.ld_in + r];
    for (int j = 0; j < jb.n - jb.k; ++j)
      acc = cfma(jb.T[(int64_t)j * jb.k + i], jb.in[(int64_t)jb.perm[jb.k + j] * jb.ld_in + r], acc);
    jb.out[(int64_t)i * jb.ld_out + r] = acc;
  }
}

// out = P^T * In  (In: n x other, out: k x other): out[i, :] = In[perm[i], :] + sum_j T[i, j] In[perm[k+j], :]
__global__ void k_left_pt(const PJob* jobs) {
  const PJob jb = jobs[blockIdx.y];
  const int64_t tot = (int64_t)jb.other * jb.k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % jb.k), c = (int)(e / jb.k);
    const cplx* col = jb.in + (int64_t)c * jb.ld_in;
    cplx acc = col[jb.perm[i]];
    for (int j = 0; j < jb.n - jb.k; ++j) acc = cfma(jb.T[(int64_t)j * jb.k + i], col[jb.perm[jb.k + j]], acc);
    jb.out[(int64_t)c * jb.ld_out + i] = acc;
  }
}

// Parent index sets from the children's skeletons: idx_p = [idx_a(perm_a[0..k_a)), idx_b(perm_b[0..k_b))].
struct GatherJob {
  int64_t src_off, dst_off;
  int k;
};
__global__ void k_gather_skel(const GatherJob* jobs, const int64_t* src_idx, const int* src_perm, int64_t* dst_idx) {
  const GatherJob jb = jobs[blockIdx.y];
  for (int i = threadIdx.x; i < jb.k; i += blockDim.x)
    dst_idx[jb.dst_off + i] = src_idx[jb.src_off + src_perm[jb.src_off + i]];
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------

// C = beta C + sum of the split-K partial products W_s (fixed order: deterministic).
struct SplitRed {
  cplx* C;
  const cplx* W;
  int m, n, ldc, splits;
  cplx beta;
};
__global__ void k_splitk_reduce(const SplitRed* reds, int nred) {
  const SplitRed r = reds[blockIdx.y];
  const int64_t tot = (int64_t)r.m * r.n, mn = tot;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % r.m);
    const int64_t j = e / r.m;
    cplx acc = cmk(0.0, 0.0);
    for (int sidx = 0; sidx < r.splits; ++sidx) acc = cadd(acc, r.W[sidx * mn + e]);
    cplx* c = r.C + j * r.ldc + i;
    if (r.beta.x != 0.0 || r.beta.y != 0.0) acc = cfma(r.beta, *c, acc);
    *c = acc;
  }
}

// Batched GEMMs.  Jobs with a long inner dimension and few output tiles (tall-skinny
// products over all N boundary nodes) are split along K so that every SM gets work; the
// partial products are summed in a fixed order by k_splitk_reduce.
static void launch_gemms(std::vector<GemmJob>& jobs_in, cudaStream_t s) {
  if (jobs_in.empty()) return;
  double fl = 0.0, by = 0.0;
  for (const auto& j : jobs_in) {
    fl += 8.0 * j.m * (double)j.n * j.k;
    by += 16.0 * ((double)j.m * j.k + (double)j.k * j.n + (double)j.m * j.n *
                  ((j.beta.x != 0.0 || j.beta.y != 0.0) ? 2.0 : 1.0));
  }
  std::vector<GemmJob> jobs;
  std::vector<SplitRed> reds;
  std::vector<size_t> red_ws_off;
  int64_t ws = 0;
  for (const auto& j : jobs_in) {
    const int64_t tiles = (int64_t)((j.m + GBM - 1) / GBM) * ((j.n + GBN - 1) / GBN);
    int splits = 1;
    if (j.k >= 8192 && tiles > 0 && tiles < 304) {
      splits = (int)std::min<int64_t>((j.k + 4095) / 4096, std::max<int64_t>(1, 1216 / tiles));
    }
    if (splits <= 1) {
      jobs.push_back(j);
      continue;
    }
    int chunk = (j.k + splits - 1) / splits;
    chunk = (chunk + GBK - 1) / GBK * GBK;
    splits = (j.k + chunk - 1) / chunk;
    SplitRed r{j.C, nullptr, j.m, j.n, j.ldc, splits, j.beta};
    reds.push_back(r);
    red_ws_off.push_back((size_t)ws);
    for (int sidx = 0; sidx < splits; ++sidx) {
      const int k0 = sidx * chunk, kl = std::min(chunk, j.k - k0);
      GemmJob sj = j;
      sj.A = j.transA ? j.A + k0 : j.A + (int64_t)k0 * j.lda;
      sj.B = j.B + k0;
      sj.k = kl;
      sj.C = nullptr;  // set below (workspace)
      sj.ldc = j.m;
      sj.beta = cmk(0.0, 0.0);
      sj.tile_base = (int)(ws + (int64_t)sidx * j.m * j.n);  // temporary: workspace offset
      jobs.push_back(sj);
    }
    ws += (int64_t)splits * j.m * j.n;
  }
  DevBuf<cplx> W(std::max<int64_t>(ws, 1));
  for (auto& j : jobs)
    if (j.C == nullptr) j.C = W.get() + j.tile_base;
  for (size_t r = 0; r < reds.size(); ++r) reds[r].W = W.get() + red_ws_off[r];
  const int64_t tiles = gemm_plan(jobs.data(), (int)jobs.size());
  if (tiles > 0) {
    DevBuf<GemmJob> dj(jobs.size());
    HBS_CUDA(cudaMemcpyAsync(dj.get(), jobs.data(), jobs.size() * sizeof(GemmJob), cudaMemcpyHostToDevice, s));
    if (gemm_double_float()) {
      prof::KScope _ks("k_zgemm_batched_df", s, fl, by);
      k_zgemm_batched_df<<<(unsigned)tiles, 256, 0, s>>>(dj.get(), (int)jobs.size());
    } else {
      prof::KScope _ks("k_zgemm_batched", s, fl, by);
      k_zgemm_batched<<<(unsigned)tiles, 256, 0, s>>>(dj.get(), (int)jobs.size());
    }
  }
  HBS_LAUNCH_CHECK("k_zgemm_batched");
  if (!reds.empty()) {
    DevBuf<SplitRed> dr(reds.size());
    HBS_CUDA(cudaMemcpyAsync(dr.get(), reds.data(), reds.size() * sizeof(SplitRed), cudaMemcpyHostToDevice, s));
    int64_t mx = 0;
    for (auto& r : reds) mx = std::max<int64_t>(mx, (int64_t)r.m * r.n);
    prof::KScope _ks("k_splitk_reduce", s);
    k_splitk_reduce<<<dim3(grid_1d(mx, 256, 1024), (unsigned)reds.size()), 256, 0, s>>>(dr.get(), (int)reds.size());
    HBS_LAUNCH_CHECK("k_splitk_reduce");
  }
  // job tables and the workspace are freed in stream order (cudaFreeAsync) after the kernels
}

void run_gemms(std::vector<GemmJob>& jobs, cudaStream_t s) { launch_gemms(jobs, s); }

template <typename J>
static DevBuf<J> upload_jobs(const std::vector<J>& v, cudaStream_t s) {
  DevBuf<J> d(v.size());
  if (!v.empty())
    HBS_CUDA(cudaMemcpyAsync(d.get(), v.data(), v.size() * sizeof(J), cudaMemcpyHostToDevice, s));
  return d;
}

static inline int grid_for(int64_t tot, int nt, int cap = 4096) {
  int64_t b = (tot + nt - 1) / nt;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

DevGeom Handle_geom(const Handle& h) {
  DevGeom g;
  g.x = h.x.get(); g.y = h.y.get(); g.nx = h.nx.get(); g.ny = h.ny.get(); g.w = h.w.get();
  g.n = h.N; g.omega = h.omega;
  return g;
}

// Work above which one matrix is decomposed by the multi-CTA kernels instead of one CTA.
static bool big_cpqr(const CpqrJob& j) { return (double)j.m * j.n * std::min(j.m, j.n) > 4e6; }
static bool big_inverse(int n) { return n > 128; }

// Batched CPQR-ID of the matrices described by `jobs` (in `pool`).  Returns ranks.
// Small matrices go to one launch with one CTA each; large ones (the top tree levels,
// where a level has few nodes) share one persistent launch on all SMs (pqr.cu).
std::vector<int> batched_id(std::vector<CpqrJob>& jobs, cplx* pool, cplx* tpool, int* permpool, double tol,
                            cudaStream_t s) {
  std::vector<int> ranks(jobs.size(), 0);
  if (jobs.empty()) return ranks;
  std::vector<CpqrJob> small;
  std::vector<size_t> small_idx, big_idx;
  // A level with at most 128 nodes runs all of them in one persistent multi-CTA launch
  // (pqr.cu): one CTA per node would leave SMs idle and serialize on its largest node.
  // With more nodes, one CTA per node keeps every SM busy, and only the large nodes (if
  // at most 128 of them) go to the persistent launch.
  size_t nbig = 0;
  for (const auto& j : jobs) nbig += big_cpqr(j) ? 1 : 0;
  const bool all_big = jobs.size() <= 128;
  const bool use_big = all_big || (nbig > 0 && nbig <= 128);
  for (size_t i = 0; i < jobs.size(); ++i) {
    if (use_big && (all_big || big_cpqr(jobs[i]))) {
      big_idx.push_back(i);
    } else {
      small_idx.push_back(i);
      small.push_back(jobs[i]);
      small.back().job = (int)(small.size() - 1);
    }
  }
  if (!small.empty()) {
    int maxn = 0;
    for (auto& j : small) maxn = std::max(maxn, j.n);
    DevBuf<CpqrJob> dj = upload_jobs(small, s);
    DevBuf<int> dr(small.size());
    size_t sm = (size_t)maxn * (2 * sizeof(double) + sizeof(int));
    if (sm > 48 * 1024)
      HBS_CUDA(cudaFuncSetAttribute(k_cpqr<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    {
      prof::KScope _ks("k_cpqr", s);
      k_cpqr<256><<<(unsigned)small.size(), 256, sm, s>>>(dj.get(), pool, tpool, permpool, dr.get(), tol, 1 << 30);
    }
    HBS_LAUNCH_CHECK("k_cpqr");
    auto r = dr.download(s);
    for (size_t t = 0; t < small.size(); ++t) ranks[small_idx[t]] = r[t];
  }
  if (!big_idx.empty()) {
    std::vector<BigQrJobSpec> specs;
    for (size_t i : big_idx) {
      const CpqrJob& j = jobs[i];
      specs.push_back({pool + j.mt_off, j.m, j.n, permpool + j.perm_off, tpool + j.t_off});
    }
    auto r = big_row_id_batched(specs, tol, s);
    for (size_t t = 0; t < big_idx.size(); ++t) ranks[big_idx[t]] = r[t];
  }
  double fl = 0.0;
  for (size_t i = 0; i < jobs.size(); ++i) {
    const double m = jobs[i].m, n = jobs[i].n, k = ranks[i];
    fl += 4.0 * (4.0 * m * n * k - 2.0 * (m + n) * k * k + 4.0 / 3.0 * k * k * k) + 4.0 * k * k * (n - k);
  }
  prof::add_work("k_cpqr", fl, 0.0);
  return ranks;
}

// Batched in-place inverses; throws on a singular block.
void batched_inverse(std::vector<InvJob>& jobs_in, cplx* pool, cudaStream_t s, const char* what) {
  std::vector<InvJob> jobs;
  std::vector<std::pair<cplx*, int>> big;
  // Same split as for the IDs: at most 128 blocks all go to the persistent multi-CTA
  // Gauss-Jordan (pgj.cu); with more, one CTA per block and the large ones (if at most
  // 128) persistent.
  size_t nbig = 0;
  for (const auto& j : jobs_in) nbig += big_inverse(j.n) ? 1 : 0;
  const bool all_big = jobs_in.size() <= 128;
  const bool use_big = all_big || (nbig > 0 && nbig <= 128);
  for (auto& j : jobs_in) {
    if (use_big && (all_big || big_inverse(j.n))) big.push_back({pool + j.a_off, j.n});
    else jobs.push_back(j);
  }
  pgj_run(big, s, what);
  if (jobs.empty()) return;
  for (size_t i = 0; i < jobs.size(); ++i) jobs[i].job = (int)i;
  int64_t piv = 0;
  for (auto& j : jobs) { j.piv_off = piv; piv += j.n; }
  DevBuf<int> dpiv(std::max<int64_t>(piv, 1));
  DevBuf<InvJob> dj = upload_jobs(jobs, s);
  DevBuf<int> flags(jobs.size());
  double fl = 0.0;
  for (auto& j : jobs) fl += 8.0 * (double)j.n * j.n * j.n;
  {
    prof::KScope _ks("k_gj_inverse", s, fl, 0.0);
    k_gj_inverse<256><<<(unsigned)jobs.size(), 256, 0, s>>>(dj.get(), pool, dpiv.get(), flags.get());
  }
  HBS_LAUNCH_CHECK("k_gj_inverse");
  auto f = flags.download(s);
  for (int v : f)
    if (v) throw Error(HBS_WARN_ILLCOND, std::string("singular block in ") + what);
}

void build_hbs(Handle& h, cudaStream_t s) {
  const int64_t N = h.N;
  const DevGeom g = Handle_geom(h);
  const double rho = h.opts.proxy_rho;
  int L = 0;
  while ((N >> L) > h.opts.leaf_size || ((N + (1LL << L) - 1) >> L) > h.opts.leaf_size) ++L;
  if (L < 1) L = 1;
  h.L = L;
  h.levels.clear();
  h.levels.resize(L + 1);
  h.max_rank = 0;
  h.factor_bytes = 0.0;
  h.apply_flops = 0.0;

  static const char* kLevelNames[] = {
      "build:level_00", "build:level_01", "build:level_02", "build:level_03", "build:level_04", "build:level_05",
      "build:level_06", "build:level_07", "build:level_08", "build:level_09", "build:level_10", "build:level_11",
      "build:level_12", "build:level_13", "build:level_14", "build:level_15", "build:level_16", "build:level_17",
      "build:level_18", "build:level_19", "build:level_20", "build:level_21", "build:level_22", "build:level_23"};
  for (int l = L; l >= 0; --l) {
    prof::Phase ph_level(kLevelNames[std::min(l, 23)], s);
    Level& lv = h.levels[l];
    lv.l = l;
    lv.count = 1 << l;
    lv.first = (1 << l) - 1;
    lv.n.assign(lv.count, 0);
    lv.off.assign(lv.count, 0);
    // ---- index sets
    if (l == L) {
      for (int j = 0; j < lv.count; ++j) {
        int64_t lo = ((int64_t)j * N) >> l, hi = ((int64_t)(j + 1) * N) >> l;
        lv.n[j] = (int)(hi - lo);
        lv.off[j] = lo;
      }
      lv.ntot = N;
      std::vector<int64_t> hidx(N);
      std::iota(hidx.begin(), hidx.end(), 0);
      lv.idx.upload(hidx, s);
    } else {
      Level& ch = h.levels[l + 1];
      int64_t o = 0;
      std::vector<GatherJob> gj;
      for (int j = 0; j < lv.count; ++j) {
        int a = 2 * j, b = 2 * j + 1;
        lv.off[j] = o;
        lv.n[j] = ch.k[a] + ch.k[b];
        gj.push_back({ch.off[a], o, ch.k[a]});
        gj.push_back({ch.off[b], o + ch.k[a], ch.k[b]});
        o += lv.n[j];
      }
      lv.ntot = o;
      lv.idx.alloc(std::max<int64_t>(o, 1));
      DevBuf<GatherJob> dg = upload_jobs(gj, s);
      {
        prof::KScope _ks("k_gather_skel", s);
        k_gather_skel<<<dim3(1, (unsigned)gj.size()), 128, 0, s>>>(dg.get(), ch.idx.get(), ch.perm.get(), lv.idx.get());
      }
      HBS_LAUNCH_CHECK("k_gather_skel");
      HBS_CUDA(cudaStreamSynchronize(s));
    }
    DevBuf<int> dn;
    DevBuf<int64_t> doff;
    {
      std::vector<int> nn(lv.n.begin(), lv.n.end());
      dn.upload(nn, s);
      doff.upload(lv.off, s);
    }

    if (l == 0) {
      // ---- root: dense inverse of [[Dhat_a, A(J_a,J_b)], [A(J_b,J_a), Dhat_b]]
      Level& ch = h.levels[1];
      h.nroot = lv.n[0];
      h.Groot.alloc((size_t)h.nroot * h.nroot);
      std::vector<DJob> dj(1);
      dj[0] = {0, 0, h.nroot, ch.k[0], 0, ch.Dhat.get() + ch.dh_off[0], ch.Dhat.get() + ch.dh_off[1]};
      DevBuf<DJob> ddj = upload_jobs(dj, s);
      {
        prof::KScope _ks("k_fill_d", s);
        k_fill_d<<<dim3(grid_for((int64_t)h.nroot * h.nroot, 256), 1), 256, 0, s>>>(g, ddj.get(), lv.idx.get(), h.Groot.get());
      }
      HBS_LAUNCH_CHECK("k_fill_d root");
      std::vector<InvJob> ij(1);
      ij[0] = {0, 0, h.nroot, 0};
      batched_inverse(ij, h.Groot.get(), s, "root block");
      h.factor_bytes += 16.0 * h.nroot * h.nroot;
      h.apply_flops += 8.0 * h.nroot * h.nroot;
      lv.k.assign(1, 0);
      break;
    }

    // ---- node circles
    lv.cx.alloc(lv.count); lv.cy.alloc(lv.count); lv.rad.alloc(lv.count);
    {
      prof::KScope _ks("k_node_circles", s);
      k_node_circles<<<lv.count, 128, 0, s>>>(h.x.get(), h.y.get(), N, l, lv.cx.get(), lv.cy.get(), lv.rad.get());
    }
    HBS_LAUNCH_CHECK("k_node_circles");
    lv.h_rad = lv.rad.download(s);
    std::vector<double> hcx = lv.cx.download(s), hcy = lv.cy.download(s);

    // ---- near lists
    DevBuf<int64_t> cnt(lv.count);
    {
      prof::KScope _ks("k_near", s);
      k_near<<<lv.count, 256, 0, s>>>(h.x.get(), h.y.get(), lv.idx.get(), lv.ntot, doff.get(), dn.get(), lv.cx.get(),
                                      lv.cy.get(), lv.rad.get(), rho, cnt.get(), nullptr, nullptr);
    }
    HBS_LAUNCH_CHECK("k_near count");
    std::vector<int64_t> hc = cnt.download(s);
    std::vector<int64_t> noff(lv.count, 0);
    int64_t ntot_near = 0;
    for (int j = 0; j < lv.count; ++j) { noff[j] = ntot_near; ntot_near += hc[j]; }
    DevBuf<int64_t> dnoff;
    dnoff.upload(noff, s);
    DevBuf<int64_t> near(std::max<int64_t>(ntot_near, 1));
    {
      prof::KScope _ks("k_near", s);
      k_near<<<lv.count, 256, 0, s>>>(h.x.get(), h.y.get(), lv.idx.get(), lv.ntot, doff.get(), dn.get(), lv.cx.get(),
                                      lv.cy.get(), lv.rad.get(), rho, cnt.get(), dnoff.get(), near.get());
    }
    HBS_LAUNCH_CHECK("k_near fill");

    // ---- ID matrices
    std::vector<YJob> yj(lv.count);
    int64_t ypool = 0;
    for (int j = 0; j < lv.count; ++j) {
      double R = rho * lv.h_rad[j];
      int np = (int)(2.0 * std::ceil(h.omega * R) + 40.0);
      np = std::max(np, h.opts.n_proxy_min);
      np = (np + 7) / 8 * 8;
      yj[j] = {ypool, lv.off[j], noff[j], lv.n[j], (int)hc[j], np, hcx[j], hcy[j], R, 2.0 * HBS_PI * R / np};
      ypool += (int64_t)(2 * hc[j] + 2 * np) * lv.n[j];
    }
    DevBuf<cplx> Y(std::max<int64_t>(ypool, 1));
    {
      DevBuf<YJob> dyj = upload_jobs(yj, s);
      {
        prof::KScope _ks("k_fill_y", s);
        k_fill_y<<<dim3(64, lv.count), 256, 0, s>>>(g, dyj.get(), lv.idx.get(), near.get(), Y.get());
      }
      HBS_LAUNCH_CHECK("k_fill_y");
      std::vector<CpqrJob> cj(lv.count);
      lv.t_off.assign(lv.count, 0);
      int64_t tpool = 0;
      for (int j = 0; j < lv.count; ++j) {
        int m = 2 * (int)hc[j] + 2 * yj[j].np;
        cj[j] = {yj[j].mt_off, tpool, lv.off[j], m, lv.n[j], j};
        lv.t_off[j] = tpool;
        tpool += (int64_t)std::min(m, lv.n[j]) * lv.n[j];
      }
      lv.T.alloc(std::max<int64_t>(tpool, 1));
      lv.perm.alloc(std::max<int64_t>(lv.ntot, 1));
      lv.k = batched_id(cj, Y.get(), lv.T.get(), lv.perm.get(), h.tol, s);
    }
    Y.release();
    for (int j = 0; j < lv.count; ++j) h.max_rank = std::max(h.max_rank, lv.k[j]);

    // ---- D blocks and their inverses
    std::vector<int64_t> d_off(lv.count);
    int64_t dpool = 0;
    for (int j = 0; j < lv.count; ++j) { d_off[j] = dpool; dpool += (int64_t)lv.n[j] * lv.n[j]; }
    DevBuf<cplx> Dinv(std::max<int64_t>(dpool, 1));
    {
      std::vector<DJob> dj(lv.count);
      for (int j = 0; j < lv.count; ++j) {
        if (l == L) {
          dj[j] = {d_off[j], lv.off[j], lv.n[j], 0, 1, nullptr, nullptr};
        } else {
          Level& ch = h.levels[l + 1];
          dj[j] = {d_off[j], lv.off[j], lv.n[j], ch.k[2 * j], 0, ch.Dhat.get() + ch.dh_off[2 * j],
                   ch.Dhat.get() + ch.dh_off[2 * j + 1]};
        }
      }
      DevBuf<DJob> ddj = upload_jobs(dj, s);
      {
        prof::KScope _ks("k_fill_d", s);
        k_fill_d<<<dim3(64, lv.count), 256, 0, s>>>(g, ddj.get(), lv.idx.get(), Dinv.get());
      }
      HBS_LAUNCH_CHECK("k_fill_d");
      std::vector<InvJob> ij(lv.count);
      for (int j = 0; j < lv.count; ++j) ij[j] = {d_off[j], 0, lv.n[j], j};
      batched_inverse(ij, Dinv.get(), s, "leaf/level block");
    }
    // X = D^{-1} P (n x k), Yt = P^T D^{-1} (k x n), S = P^T X (k x k)
    lv.e_off.assign(lv.count, 0); lv.f_off.assign(lv.count, 0); lv.g_off.assign(lv.count, 0); lv.dh_off.assign(lv.count, 0);
    int64_t eo = 0, go = 0, dho = 0;
    for (int j = 0; j < lv.count; ++j) {
      lv.e_off[j] = eo; lv.f_off[j] = eo; eo += (int64_t)lv.n[j] * lv.k[j];
      lv.g_off[j] = go; go += (int64_t)lv.n[j] * lv.n[j];
      lv.dh_off[j] = dho; dho += (int64_t)lv.k[j] * lv.k[j];
    }
    DevBuf<cplx> X(std::max<int64_t>(eo, 1)), Yp(std::max<int64_t>(eo, 1)), S(std::max<int64_t>(dho, 1));
    {
      std::vector<PJob> rp(lv.count), lp(lv.count);
      for (int j = 0; j < lv.count; ++j) {
        const int n = lv.n[j], k = lv.k[j];
        const int* pm = lv.perm.get() + lv.off[j];
        const cplx* T = lv.T.get() + lv.t_off[j];
        rp[j] = {Dinv.get() + d_off[j], X.get() + lv.e_off[j], pm, T, n, k, n, n, n};
        lp[j] = {Dinv.get() + d_off[j], Yp.get() + lv.f_off[j], pm, T, n, k, n, n, k};
      }
      DevBuf<PJob> drp = upload_jobs(rp, s), dlp = upload_jobs(lp, s);
      {
        prof::KScope _ks("k_right_p", s);
        k_right_p<<<dim3(32, lv.count), 256, 0, s>>>(drp.get());
      }
      HBS_LAUNCH_CHECK("k_right_p");
      {
        prof::KScope _ks("k_left_pt", s);
        k_left_pt<<<dim3(32, lv.count), 256, 0, s>>>(dlp.get());
      }
      HBS_LAUNCH_CHECK("k_left_pt");
      for (int j = 0; j < lv.count; ++j) {
        const int n = lv.n[j], k = lv.k[j];
        lp[j] = {X.get() + lv.e_off[j], S.get() + lv.dh_off[j], lv.perm.get() + lv.off[j], lv.T.get() + lv.t_off[j],
                 n, k, k, n, k};
      }
      DevBuf<PJob> dlp2 = upload_jobs(lp, s);
      {
        prof::KScope _ks("k_left_pt", s);
        k_left_pt<<<dim3(32, lv.count), 256, 0, s>>>(dlp2.get());
      }
      HBS_LAUNCH_CHECK("k_left_pt S");
      HBS_CUDA(cudaStreamSynchronize(s));
    }
    // Dhat = S^{-1}
    {
      std::vector<InvJob> ij;
      for (int j = 0; j < lv.count; ++j)
        if (lv.k[j] > 0) ij.push_back({lv.dh_off[j], 0, lv.k[j], j});
      batched_inverse(ij, S.get(), s, "skeleton block P^T D^-1 P");
    }
    lv.Dhat = std::move(S);
    lv.E.alloc(std::max<int64_t>(eo, 1));
    lv.F.alloc(std::max<int64_t>(eo, 1));
    lv.G = std::move(Dinv);
    lv.g_off = d_off;
    {
      std::vector<GemmJob> gj;
      for (int j = 0; j < lv.count; ++j) {
        const int n = lv.n[j], k = lv.k[j];
        if (k == 0) continue;
        // E = X Dhat  (n x k)
        gj.push_back({X.get() + lv.e_off[j], lv.Dhat.get() + lv.dh_off[j], lv.E.get() + lv.e_off[j], n, k, k, n, k, n,
                      cmk(1, 0), cmk(0, 0), 0, 0, 0});
        // F* = Dhat Yt  (k x n)
        gj.push_back({lv.Dhat.get() + lv.dh_off[j], Yp.get() + lv.f_off[j], lv.F.get() + lv.f_off[j], k, n, k, k, k, k,
                      cmk(1, 0), cmk(0, 0), 0, 0, 0});
      }
      launch_gemms(gj, s);
      gj.clear();
      for (int j = 0; j < lv.count; ++j) {
        const int n = lv.n[j], k = lv.k[j];
        if (k == 0) continue;
        // G = D^{-1} - E Yt
        gj.push_back({lv.E.get() + lv.e_off[j], Yp.get() + lv.f_off[j], lv.G.get() + lv.g_off[j], n, n, k, n, k, n,
                      cmk(-1, 0), cmk(1, 0), 0, 0, 0});
      }
      launch_gemms(gj, s);
    }
    for (int j = 0; j < lv.count; ++j) {
      const double n = lv.n[j], k = lv.k[j];
      h.factor_bytes += 16.0 * (2 * n * k + n * n);
      h.apply_flops += 8.0 * (2 * n * k + n * n);
    }
  }
}

// x = A^{-1} b through the telescoping factorization (Sec. 4): upward b^_tau = F*_tau b_tau,
// root solve, downward x_tau = E_tau x^_tau + G_tau b_tau.
// x = A^{-1} b (trans = false) or x = A^{-T} b (trans = true, the factors transposed:
// A^{-T} = F*^T (M~ + Dhat)^{-T} E^T + G^T, applied with the same telescoping sweep).
static void apply_impl(const Handle& H, const cplx* b, cplx* xout, int64_t nrhs, cudaStream_t s, bool trans) {
  if (nrhs <= 0) return;
  const int Lv = H.L;
  const auto& levels = H.levels;
  // level vectors: up[l] holds b_tau for all nodes of level l (ntot x nrhs, ld = ntot)
  std::vector<DevBuf<cplx>> up(Lv + 1), dn(Lv + 1);
  for (int l = 0; l < Lv; ++l) {
    up[l].alloc(std::max<int64_t>(levels[l].ntot * nrhs, 1));
    dn[l].alloc(std::max<int64_t>(levels[l].ntot * nrhs, 1));
  }
  auto upptr = [&](int l) -> const cplx* { return l == Lv ? b : up[l].get(); };
  const int ta = trans ? 1 : 0;
  for (int l = Lv; l >= 1; --l) {
    const Level& lv = levels[l];
    const Level& pa = levels[l - 1];
    std::vector<GemmJob> gj;
    for (int j = 0; j < lv.count; ++j) {
      const int n = lv.n[j], k = lv.k[j];
      if (k == 0) continue;
      const int parent = j >> 1;
      const int64_t prow = pa.off[parent] + ((j & 1) ? levels[l].k[j - 1] : 0);
      // upward: F* (k x n), or E^T with E stored n x k
      const cplx* Aop = trans ? lv.E.get() + lv.e_off[j] : lv.F.get() + lv.f_off[j];
      const int lda = trans ? n : k;
      gj.push_back({Aop, upptr(l) + lv.off[j], up[l - 1].get() + prow, k, (int)nrhs, n, lda, (int)lv.ntot,
                    (int)pa.ntot, cmk(1, 0), cmk(0, 0), 0, 0, 0, ta});
    }
    run_gemms(gj, s);
  }
  {
    std::vector<GemmJob> gj(1);
    gj[0] = {H.Groot.get(), up[0].get(), dn[0].get(), H.nroot, (int)nrhs, H.nroot, H.nroot, H.nroot, H.nroot,
             cmk(1, 0), cmk(0, 0), 0, 0, 0, ta};
    run_gemms(gj, s);
  }
  for (int l = 1; l <= Lv; ++l) {
    const Level& lv = levels[l];
    const Level& pa = levels[l - 1];
    cplx* outp = l == Lv ? xout : dn[l].get();
    std::vector<GemmJob> gj;
    for (int j = 0; j < lv.count; ++j) {
      const int n = lv.n[j];
      // x_tau = G b_tau  (or G^T b_tau)
      gj.push_back({lv.G.get() + lv.g_off[j], upptr(l) + lv.off[j], outp + lv.off[j], n, (int)nrhs, n, n,
                    (int)lv.ntot, (int)lv.ntot, cmk(1, 0), cmk(0, 0), 0, 0, 0, ta});
    }
    run_gemms(gj, s);
    gj.clear();
    for (int j = 0; j < lv.count; ++j) {
      const int n = lv.n[j], k = lv.k[j];
      if (k == 0) continue;
      const int parent = j >> 1;
      const int64_t prow = pa.off[parent] + ((j & 1) ? levels[l].k[j - 1] : 0);
      // x_tau += E x^_tau  (or F*^T x^_tau with F* stored k x n)
      const cplx* Aop = trans ? lv.F.get() + lv.f_off[j] : lv.E.get() + lv.e_off[j];
      const int lda = trans ? k : n;
      gj.push_back({Aop, dn[l - 1].get() + prow, outp + lv.off[j], n, (int)nrhs, k, lda, (int)pa.ntot, (int)lv.ntot,
                    cmk(1, 0), cmk(1, 0), 0, 0, 0, ta});
    }
    run_gemms(gj, s);
  }
}

void Handle::apply_inverse(const cplx* b, cplx* xout, int64_t nrhs, cudaStream_t s) const {
  apply_impl(*this, b, xout, nrhs, s, false);
}

void Handle::apply_inverse_transpose(const cplx* b, cplx* xout, int64_t nrhs, cudaStream_t s) const {
  apply_impl(*this, b, xout, nrhs, s, true);
}

}  // namespace hbs
