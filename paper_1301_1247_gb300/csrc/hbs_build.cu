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
#include "tune.hpp"
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

// One node of one solver's level: its original points [lo, hi) and where its circle goes.
struct CircleJob {
  const double* x;
  const double* y;
  int64_t lo, hi;
  double* out;  // cx, cy, radius
};

// Enclosing circle of the original points of each node (one block per job): centre of the
// bounding box, radius = largest distance from it.
__global__ void k_node_circles(const CircleJob* jobs) {
  __shared__ double red[32];
  const CircleJob jb = jobs[blockIdx.x];
  const double* x = jb.x;
  const double* y = jb.y;
  const int64_t lo = jb.lo, hi = jb.hi;
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
    jb.out[0] = ccx;
    jb.out[1] = ccy;
    jb.out[2] = sqrt(r);
  }
}

// Near lists: active points of other nodes of the level (same solver) inside a node's
// proxy circle.  One block per node scans, in increasing position, the ranges of the level's
// active points that belong to candidate nodes (those whose enclosing circle meets the proxy
// circle: no point of another node can be near), so the list order is deterministic and the
// same as a scan of every point.  With `out` == nullptr only the count is produced.
struct NearJob {
  const double* x;
  const double* y;
  const int64_t* idx;       // the level's active points
  const longlong2* ranges;  // position ranges [x, y) in idx to scan, increasing, the node's own excluded
  int nranges;
  double cx, cy, R2;
  int64_t* count;           // one element
  int64_t* out;             // the node's near list, or nullptr
};

__global__ void k_near(const NearJob* jobs) {
  __shared__ int wsum[32];
  __shared__ int64_t base;
  const NearJob jb = jobs[blockIdx.x];
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int rg = 0; rg < jb.nranges; ++rg)
  for (int64_t p0 = jb.ranges[rg].x; p0 < jb.ranges[rg].y; p0 += blockDim.x) {
    const int64_t p = p0 + threadIdx.x;
    bool f = false;
    int64_t g = 0;
    if (p < jb.ranges[rg].y) {
      g = jb.idx[p];
      const double ddx = jb.x[g] - jb.cx, ddy = jb.y[g] - jb.cy;
      f = ddx * ddx + ddy * ddy < jb.R2;
    }
    const unsigned b = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[warp] = __popc(b);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) before += wsum[w];
      total += wsum[w];
    }
    if (f && jb.out) jb.out[base + before + __popc(b & ((1u << lane) - 1u))] = g;
    __syncthreads();
    if (threadIdx.x == 0) base += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *jb.count = base;
}

struct YJob {
  DevGeom g;           // the solver's geometry
  const int64_t* idx;  // the node's active points (n)
  const int64_t* near; // the node's near list (nn)
  cplx* mt;            // output Mt (m x n, m = 2 nn + 2 np)
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
// Dynamic shared memory: 4 np doubles (the node's proxy points and their directions,
// formed once per block instead of once per entry).
__global__ void k_fill_y(const YJob* jobs) {
  extern __shared__ double sprox[];
  const YJob jb = jobs[blockIdx.y];
  const DevGeom& g = jb.g;
  if (g.comps != 1) return;
  double* pxs = sprox;
  double* pys = sprox + jb.np;
  double* pcs = sprox + 2 * jb.np;
  double* psn = sprox + 3 * jb.np;
  for (int p = threadIdx.x; p < jb.np; p += blockDim.x) {
    const double th = 2.0 * HBS_PI * (double)p / (double)jb.np;
    double sn, cs;
    sincos(th, &sn, &cs);
    pxs[p] = jb.cx + jb.R * cs;
    pys[p] = jb.cy + jb.R * sn;
    pcs[p] = cs;
    psn[p] = sn;
  }
  __syncthreads();
  const int m = 2 * jb.nn + 2 * jb.np;
  const int half = jb.nn + jb.np;
  const int64_t tot = (int64_t)half * jb.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % half), c = (int)(e / half);
    const int64_t gj = jb.idx[c];
    cplx* col = jb.mt + (int64_t)c * m;
    const double xj = g.x[gj], yj = g.y[gj];
    if (r < jb.nn) {
      const int64_t gi = jb.near[r];
      cplx v1, v2;
      if (gi == gj) {
        v1 = v2 = cmk(0.5, 0.0);
      } else {
        const double dx = g.x[gi] - xj, dy = g.y[gi] - yj;
        const double rr = sqrt(dx * dx + dy * dy);
        cplx h0, h1;
        hankel01(g.omega * rr, &h0, &h1, g.df);
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
      const double cs = pcs[p], sn = psn[p];
      const double px = pxs[p], py = pys[p];
      const double dx = xj - px, dy = yj - py;
      const double rr = sqrt(dx * dx + dy * dy);
      cplx h0, h1;
      hankel01(g.omega * rr, &h0, &h1, g.df);
      const double q = 0.25 * g.omega / rr;
      // combined-layer source at the proxy (normal = radial direction), target node j
      col[2 * jb.nn + p] = cscale(combined_from(q * (dx * cs + dy * sn), h0, h1, g.omega), jb.wp);
      // field at the proxy of the node's source j
      col[2 * jb.nn + jb.np + p] =
          cscale(combined_from(-q * (dx * g.nx[gj] + dy * g.ny[gj]), h0, h1, g.omega), g.w[gj]);
    }
  }
}

// Rows of Mt per node: 2 nn near rows, then np proxy rows per direction and wavenumber
// (one wavenumber for sound-soft obstacles, the outside and the inside one for the
// transmission problem).
__host__ __device__ __forceinline__ int y_rows(const YJob& y) { return 2 * y.nn + 2 * y.np * y.g.comps; }

// The transmission problem's Mt (Sec. 5): columns are the node's unknowns, rows
// A(near_r, j) and A(j, near_r) (r < nn), then for each wavenumber k of (w, n w) the
// combined-layer proxy sources at k acting on the row of unknown j (outside -> in), then
// for each k the field at the proxy points of unknown j's layer at k (in -> out).  Every
// far interaction of the operator is a sum of fields of the two wavenumbers, each a
// Helmholtz field in the proxy disk (in) or a radiating one determined by its values on the
// circle (out), so the proxies of both wavenumbers span it.
__global__ void k_fill_y_tr(const YJob* jobs) {
  extern __shared__ double sprox[];
  const YJob jb = jobs[blockIdx.y];
  const DevGeom& g = jb.g;
  if (g.comps != 2) return;
  double* pxs = sprox;
  double* pys = sprox + jb.np;
  double* pcs = sprox + 2 * jb.np;
  double* psn = sprox + 3 * jb.np;
  for (int p = threadIdx.x; p < jb.np; p += blockDim.x) {
    const double th = 2.0 * HBS_PI * (double)p / (double)jb.np;
    double sn, cs;
    sincos(th, &sn, &cs);
    pxs[p] = jb.cx + jb.R * cs;
    pys[p] = jb.cy + jb.R * sn;
    pcs[p] = cs;
    psn[p] = sn;
  }
  __syncthreads();
  const int m = 2 * jb.nn + 4 * jb.np;
  const int half = jb.nn + 2 * jb.np;
  const int64_t tot = (int64_t)half * jb.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % half), c = (int)(e / half);
    const int64_t gj = jb.idx[c];
    cplx* col = jb.mt + (int64_t)c * m;
    if (r < jb.nn) {
      const int64_t gi = jb.near[r];
      cplx v1, v2;
      if ((gi >> 1) == (gj >> 1)) {  // the node's own 2 x 2 block: the identity
        v1 = v2 = cmk(gi == gj ? 1.0 : 0.0, 0.0);
      } else {
        tr_a_entry_pair(g, gi, gj, &v1, &v2);
      }
      col[r] = v1;
      col[jb.nn + r] = v2;
    } else {
      const int p = r - jb.nn;
      const int q = p % jb.np;
      const double k = p < jb.np ? g.omega : g.omega_in;
      cplx row, field;
      proxy_pair_entries(g, gj, pxs[q], pys[q], pcs[q], psn[q], k, &row, &field);
      col[2 * jb.nn + p] = cscale(row, jb.wp);
      col[2 * jb.nn + 2 * jb.np + p] = cscale(field, g.w[gj]);
    }
  }
}

// Rows of a randomized ID sketch beyond the node's size (l = n + kSketchOver).
constexpr int kSketchOver = 16;

// Omega (l x m, ld = l): independent random signs +-1 from SplitMix64 (Steele, Lea and Flood,
// 2014) of the entry's position, the same matrix on every call.
__global__ void k_sketch_signs(cplx* om, int l, int m) {
  const int64_t tot = (int64_t)l * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = (uint64_t)e + 0x2545F4914F6CDD1Dull;
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    om[e] = cmk((z & 1) ? 1.0 : -1.0, 0.0);
  }
}

struct DJob {
  DevGeom g;           // the solver's geometry
  const int64_t* idx;  // the node's active points (n)
  cplx* d;             // output (n x n)
  int n, k0;           // node size; first child's skeleton size (0 for leaves)
  int leaf;
  const cplx* dh0;     // children's Dhat (k0 x k0, k1 x k1)
  const cplx* dh1;
};

__global__ void k_fill_d(const DJob* jobs) {
  const DJob jb = jobs[blockIdx.y];
  const DevGeom& g = jb.g;
  const int64_t* idx = jb.idx;
  const int n = jb.n;
  const int64_t tot = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % n), c = (int)(e / n);
    cplx v;
    if (jb.leaf) {
      v = a_entry(g, idx[r], idx[c]);
    } else {
      const int k0 = jb.k0, k1 = n - k0;
      const bool r0 = r < k0, c0 = c < k0;
      if (r0 && c0) v = jb.dh0[(int64_t)c * k0 + r];
      else if (!r0 && !c0) v = jb.dh1[(int64_t)(c - k0) * k1 + (r - k0)];
      else v = a_entry(g, idx[r], idx[c]);
    }
    jb.d[e] = v;
  }
}

// Permuted copies for the products with P = Pi [I; T^T] (Pi: the ID's column order):
//   cols: out(:, c) = in(:, perm[c]) (rows x n), first = out(:, 0..k)   (ld rows)
//   rows: out(r, :) = in(perm[r], :) (n x cols), first = out(0..k, :)   (ld k)
// and Tt = T^T ((n - k) x k).  The rest of each product is then a GEMM with T or T^T.
struct PermJob {
  const cplx* in;
  cplx* out;
  cplx* first;
  const int* perm;
  const cplx* T;
  cplx* Tt;
  int n, k, other, ld_in;
  int by_rows;
};
__global__ void k_perm_copy(const PermJob* jobs) {
  const PermJob jb = jobs[blockIdx.y];
  const int64_t tot = (int64_t)jb.n * jb.other;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    if (jb.by_rows) {  // out is n x other
      const int r = (int)(e % jb.n), c = (int)(e / jb.n);
      const cplx v = jb.in[(int64_t)c * jb.ld_in + jb.perm[r]];
      jb.out[e] = v;
      if (r < jb.k) jb.first[(int64_t)c * jb.k + r] = v;
    } else {  // out is other x n
      const int r = (int)(e % jb.other), c = (int)(e / jb.other);
      const cplx v = jb.in[(int64_t)jb.perm[c] * jb.ld_in + r];
      jb.out[e] = v;
      if (c < jb.k) jb.first[e] = v;
    }
  }
  if (jb.Tt != nullptr) {
    const int nk = jb.n - jb.k;
    const int64_t tt = (int64_t)nk * jb.k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tt; e += (int64_t)gridDim.x * blockDim.x) {
      const int j = (int)(e % nk), i = (int)(e / nk);
      jb.Tt[e] = jb.T[(int64_t)j * jb.k + i];  // Tt(j, i) = T(i, j)
    }
  }
}

// Parent index sets from the children's skeletons: idx_p = [idx_a(perm_a[0..k_a)), idx_b(perm_b[0..k_b))].
struct GatherJob {
  const int64_t* src_idx;  // the child's active points
  const int* src_perm;     // the child's pivot order
  int64_t* dst;
  int k;
};
__global__ void k_gather_skel(const GatherJob* jobs) {
  const GatherJob jb = jobs[blockIdx.y];
  for (int i = threadIdx.x; i < jb.k; i += blockDim.x) jb.dst[i] = jb.src_idx[jb.src_perm[i]];
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
  int transC;
};
__global__ void k_splitk_reduce(const SplitRed* reds, int nred) {
  const SplitRed r = reds[blockIdx.y];
  const int64_t tot = (int64_t)r.m * r.n, mn = tot;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % r.m);
    const int64_t j = e / r.m;
    cplx acc = cmk(0.0, 0.0);
    for (int sidx = 0; sidx < r.splits; ++sidx) acc = cadd(acc, r.W[sidx * mn + e]);
    cplx* c = r.transC ? r.C + (int64_t)i * r.ldc + j : r.C + j * r.ldc + i;
    if (r.beta.x != 0.0 || r.beta.y != 0.0) acc = cfma(r.beta, *c, acc);
    *c = acc;
  }
}

// Batched GEMMs.  Jobs with a long inner dimension and few output tiles (tall-skinny
// products over all N boundary nodes) are split along K so that every SM gets work; the
// partial products are summed in a fixed order by k_splitk_reduce.
static void launch_gemms(std::vector<GemmJob>& jobs_all, cudaStream_t s) {
  if (jobs_all.empty()) return;
  // large products on the tensor cores when the thread's mode asks for it
  std::vector<GemmJob> jobs_in, jobs_tc;
  for (const auto& j : jobs_all) {
    if (gemm_tensor() && ozaki_eligible(j)) jobs_tc.push_back(j);
    else jobs_in.push_back(j);
  }
  ozaki_gemm_batched(jobs_tc, s);
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
    SplitRed r{j.C, nullptr, j.m, j.n, j.ldc, splits, j.beta, j.transC};
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
      sj.transC = 0;  // partial products in the column-major workspace
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


DevGeom Handle_geom(const Handle& h) {
  DevGeom g;
  g.x = h.x.get(); g.y = h.y.get(); g.nx = h.nx.get(); g.ny = h.ny.get(); g.w = h.w.get();
  g.n = h.N; g.omega = h.omega;
  g.comps = h.comps;
  g.omega_in = h.index * h.omega;
  // double-float Hankel series in the thread's double-float mode; the transmission
  // operator's kernel differences cancel their leading singular terms, so their Hankel
  // functions stay in FP64
  g.df = h.comps == 2 ? false : gemm_double_float();
  return g;
}

// Work above which one matrix is decomposed by the multi-CTA kernels instead of one CTA.
static bool big_cpqr(const CpqrJob& j) { return (double)j.m * j.n * std::min(j.m, j.n) > 4e6; }
static bool big_inverse(int n) { return n > 128; }

// Largest root (sum of the level-2 skeletons) for which level 1 is left uncompressed.  At the
// top of the tree the level-1 ID and inversions are latency-bound work on two nodes; without
// them the root inverts the level-2 skeletons' coupled system directly (the same system,
// one interpolative decomposition fewer).
constexpr int kPassThroughRootMax = 2048;

static bool passthrough_level(const Handle& h, int l) {
  if (l != 1 || h.L < 2) return false;
  const Level& lv = h.levels[1];
  return lv.n.size() == 2 && lv.n[0] + lv.n[1] <= kPassThroughRootMax;
}

// Batched CPQR-ID of the matrices described by `jobs`.  Returns ranks.
// Small matrices go to one launch with one CTA each; large ones (the top tree levels,
// where a level has few nodes) share one persistent launch on all SMs (pqr.cu).
std::vector<int> batched_id(std::vector<CpqrJob>& jobs, double tol, cudaStream_t s) {
  std::vector<int> ranks(jobs.size(), 0);
  if (jobs.empty()) return ranks;
  std::vector<CpqrJob> small;
  std::vector<size_t> small_idx, big_idx;
  // A level with at most 128 nodes runs all of them in one persistent multi-CTA launch
  // (pqr.cu): one CTA per node would leave SMs idle and serialize on its largest node (at
  // N = 10^5 the 128-node level took 80 ms that way against 28 ms in the persistent
  // launch).  With more nodes, one CTA per node keeps every SM busy, and only the large
  // nodes (if at most 128 of them) go to the persistent launch.
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
    // double-float updates on handles built with double-float precision
    const bool df = gemm_double_float();
    HBS_CUDA(raise_smem_limit(df ? (const void*)k_cpqr<256, true> : (const void*)k_cpqr<256, false>, sm));
    {
      prof::KScope _ks("k_cpqr", s);
      if (df) k_cpqr<256, true><<<(unsigned)small.size(), 256, sm, s>>>(dj.get(), dr.get(), tol, 1 << 30);
      else k_cpqr<256, false><<<(unsigned)small.size(), 256, sm, s>>>(dj.get(), dr.get(), tol, 1 << 30);
    }
    HBS_LAUNCH_CHECK("k_cpqr");
    auto r = dr.download(s);
    for (size_t t = 0; t < small.size(); ++t) ranks[small_idx[t]] = r[t];
  }
  if (!big_idx.empty()) {
    std::vector<BigQrJobSpec> specs;
    for (size_t i : big_idx) {
      const CpqrJob& j = jobs[i];
      specs.push_back({j.mt, j.m, j.n, j.perm, j.t});
    }
    auto r = big_row_id_batched(specs, tol, s);
    for (size_t t = 0; t < big_idx.size(); ++t) ranks[big_idx[t]] = r[t];
  }
  // algorithmic work of an interpolative decomposition of an m x n block of rank k: 8 m n k
  // flops (the Householder factorization executes about twice that), and the block read
  // once plus the interpolation matrix and the order written once
  double fl = 0.0, by = 0.0;
  for (size_t i = 0; i < jobs.size(); ++i) {
    const double m = jobs[i].m, n = jobs[i].n, k = ranks[i];
    fl += 8.0 * m * n * k;
    by += 16.0 * m * n + 16.0 * k * (n - k) + 4.0 * n;
  }
  prof::add_work("k_cpqr", fl, by);
  return ranks;
}

// Batched in-place inverses; throws on a singular block.
void batched_inverse(std::vector<InvJob>& jobs_in, cudaStream_t s, const char* what) {
  std::vector<InvJob> jobs;
  std::vector<std::pair<cplx*, int>> big;
  // Same split as for the IDs: at most 128 blocks all go to one multi-CTA launch; with
  // more, one CTA per block and the large ones (if at most 128) multi-CTA.
  size_t nbig = 0;
  for (const auto& j : jobs_in) nbig += big_inverse(j.n) ? 1 : 0;
  const bool all_big = jobs_in.size() <= 128;
  const bool use_big = all_big || (nbig > 0 && nbig <= 128);
  for (auto& j : jobs_in) {
    if (use_big && (all_big || big_inverse(j.n))) big.push_back({j.a, j.n});
    else jobs.push_back(j);
  }
  if (!big.empty()) {
    // The multi-CTA inversion: the persistent Gauss-Jordan (pgj.cu, one grid barrier per
    // column step; the default) or the blocked one (bgj.cu) on clusters of 1, 2, 4 or 8 CTAs
    // per block; the autotuner measures them per shape class when it is on.
    int nmax = 0;
    for (const auto& m : big) nmax = std::max(nmax, m.second);
    int n_pow = 1, c_pow = 1;
    while (n_pow < nmax) n_pow *= 2;
    while (c_pow < (int)big.size()) c_pow *= 2;
    const std::string tkey = "inverse/n" + std::to_string(n_pow) + "/j" + std::to_string(c_pow) +
                             (gemm_double_float() ? "/df" : "");
    static const int kCs[5] = {0, 1, 2, 4, 8};
    int var = tune::choose(tkey, 5, 0);
    if (var > 0 && bgj_panel_width(nmax, kCs[var]) == 0) {  // does not fit: not a candidate
      if (tune::exploring(tkey, 5)) tune::record(tkey, var, 5, 1e30f);
      var = 0;
    }
    bool done = false;
    if (var > 0) {
      try {
        tune::Timed timed(tkey, var, 5, s);
        bgj_run(big, kCs[var], s, what);
        done = true;
      } catch (const Error& e) {
        if (!bgj_unavailable(e)) throw;
        tune::record(tkey, var, 5, 1e30f);  // this shape cannot run here: never choose it
      }
    }
    if (!done) {
      tune::Timed timed(tkey, 0, 5, s);
      pgj_run(big, s, what);
    }
  }
  if (jobs.empty()) return;
  for (size_t i = 0; i < jobs.size(); ++i) jobs[i].job = (int)i;
  int64_t piv = 0;
  for (auto& j : jobs) piv += j.n;
  DevBuf<int> dpiv(std::max<int64_t>(piv, 1));
  piv = 0;
  for (auto& j : jobs) { j.piv = dpiv.get() + piv; piv += j.n; }
  DevBuf<InvJob> dj = upload_jobs(jobs, s);
  DevBuf<int> flags(jobs.size());
  double fl = 0.0;
  for (auto& j : jobs) fl += 8.0 * (double)j.n * j.n * j.n;
  {
    prof::KScope _ks("k_gj_inverse", s, fl, 0.0);
    // double-float eliminations on handles built with double-float precision
    if (gemm_double_float()) k_gj_inverse<256, true><<<(unsigned)jobs.size(), 256, 0, s>>>(dj.get(), flags.get());
    else k_gj_inverse<256, false><<<(unsigned)jobs.size(), 256, 0, s>>>(dj.get(), flags.get());
  }
  HBS_LAUNCH_CHECK("k_gj_inverse");
  auto f = flags.download(s);
  for (int v : f)
    if (v) throw Error(HBS_WARN_ILLCOND, std::string("singular block in ") + what);
}

// Launches a per-job kernel whose job index is blockIdx.y, in chunks that respect the
// 65535 limit of gridDim.y.
template <typename J, typename F>
static void launch_jobs_y(const DevBuf<J>& dj, size_t njobs, F&& launch) {
  for (size_t j0 = 0; j0 < njobs; j0 += 65535)
    launch(dj.get() + j0, (unsigned)std::min<size_t>(65535, njobs - j0));
}

// One level of one solver processed in a stage of the (multi-solver) build.
struct LevelTask {
  Handle* h;
  int l;
  DevGeom g;
};

// HBS compression and inversion of several solvers at once.  Stage t processes level
// L_i - t of every solver i (leaves first, each tree's root last), and every kernel of a
// stage covers all nodes of all its solvers' levels: one launch per kernel and stage,
// whatever the number of solvers.
void build_hbs_multi(const std::vector<Handle*>& hs, cudaStream_t s) {
  int Lmax = 0;
  for (Handle* hp : hs) {
    Handle& h = *hp;
    int L = 0;
    while ((h.N >> L) > h.opts.leaf_size || ((h.N + (1LL << L) - 1) >> L) > h.opts.leaf_size) ++L;
    if (L < 1) L = 1;
    h.L = L;
    h.levels.clear();
    h.levels.resize(L + 1);
    h.max_rank = 0;
    h.factor_bytes = 0.0;
    h.apply_flops = 0.0;
    Lmax = std::max(Lmax, L);
  }
  static const char* kLevelNames[] = {
      "build:level_00", "build:level_01", "build:level_02", "build:level_03", "build:level_04", "build:level_05",
      "build:level_06", "build:level_07", "build:level_08", "build:level_09", "build:level_10", "build:level_11",
      "build:level_12", "build:level_13", "build:level_14", "build:level_15", "build:level_16", "build:level_17",
      "build:level_18", "build:level_19", "build:level_20", "build:level_21", "build:level_22", "build:level_23"};
  for (int t = 0; t <= Lmax; ++t) {
    prof::Phase ph_level(kLevelNames[std::min(Lmax - t, 23)], s);
    std::vector<LevelTask> tasks, roots;
    for (Handle* hp : hs) {
      const int l = hp->L - t;
      if (l < 0) continue;
      (l == 0 ? roots : tasks).push_back({hp, l, Handle_geom(*hp)});
    }
    // ---- index sets
    {
      std::vector<GatherJob> gj;
      auto index_sets = [&](LevelTask& tk) {
        Handle& h = *tk.h;
        const int l = tk.l;
        Level& lv = h.levels[l];
        lv.l = l;
        lv.count = 1 << l;
        lv.first = (1 << l) - 1;
        lv.n.assign(lv.count, 0);
        lv.off.assign(lv.count, 0);
        if (l == h.L) {
          for (int j = 0; j < lv.count; ++j) {
            const int64_t lo = ((int64_t)j * h.N) >> l, hi = ((int64_t)(j + 1) * h.N) >> l;
            lv.n[j] = (int)(hi - lo);
            lv.off[j] = lo;
          }
          lv.ntot = h.N;
          std::vector<int64_t> hidx(h.N);
          std::iota(hidx.begin(), hidx.end(), 0);
          lv.idx.upload(hidx, s);
        } else {
          Level& ch = h.levels[l + 1];
          int64_t o = 0;
          for (int j = 0; j < lv.count; ++j) {
            lv.off[j] = o;
            lv.n[j] = ch.k[2 * j] + ch.k[2 * j + 1];
            o += lv.n[j];
          }
          lv.ntot = o;
          lv.idx.alloc(std::max<int64_t>(o, 1));
          for (int j = 0; j < lv.count; ++j) {
            const int a = 2 * j, b = 2 * j + 1;
            gj.push_back({ch.idx.get() + ch.off[a], ch.perm.get() + ch.off[a], lv.idx.get() + lv.off[j], ch.k[a]});
            gj.push_back({ch.idx.get() + ch.off[b], ch.perm.get() + ch.off[b], lv.idx.get() + lv.off[j] + ch.k[a],
                          ch.k[b]});
          }
        }
      };
      for (auto& tk : tasks) index_sets(tk);
      for (auto& tk : roots) index_sets(tk);
      if (!gj.empty()) {
        DevBuf<GatherJob> dg = upload_jobs(gj, s);
        prof::KScope _ks("k_gather_skel", s);
        launch_jobs_y(dg, gj.size(), [&](const GatherJob* p, unsigned ny) { k_gather_skel<<<dim3(1, ny), 128, 0, s>>>(p); });
        HBS_LAUNCH_CHECK("k_gather_skel");
      }
    }

    // ---- roots: dense inverse of [[Dhat_a, A(J_a,J_b)], [A(J_b,J_a), Dhat_b]]
    if (!roots.empty()) {
      std::vector<DJob> dj;
      std::vector<InvJob> ij;
      for (auto& tk : roots) {
        Handle& h = *tk.h;
        Level& lv = h.levels[0];
        Level& ch = h.levels[1];
        h.nroot = lv.n[0];
        h.Groot.alloc(std::max<int64_t>((int64_t)h.nroot * h.nroot, 1));
        dj.push_back({tk.g, lv.idx.get(), h.Groot.get(), h.nroot, ch.k[0], 0, ch.Dhat.get() + ch.dh_off[0],
                      ch.Dhat.get() + ch.dh_off[1]});
        if (h.nroot > 0) ij.push_back({h.Groot.get(), nullptr, h.nroot, (int)ij.size()});
        h.factor_bytes += 16.0 * h.nroot * h.nroot;
        h.apply_flops += 8.0 * h.nroot * h.nroot;
        lv.k.assign(1, 0);
      }
      DevBuf<DJob> ddj = upload_jobs(dj, s);
      {
        prof::KScope _ks("k_fill_d", s);
        launch_jobs_y(ddj, dj.size(), [&](const DJob* p, unsigned ny) { k_fill_d<<<dim3(64, ny), 256, 0, s>>>(p); });
      }
      HBS_LAUNCH_CHECK("k_fill_d root");
      batched_inverse(ij, s, "root block");
    }
    // ---- uncompressed levels: D only, which is also Dhat; identity order, no T, E, F*, G
    {
      std::vector<LevelTask> rest;
      std::vector<DJob> dj;
      std::vector<Level*> plv;
      for (auto& tk : tasks) {
        Handle& h = *tk.h;
        if (!passthrough_level(h, tk.l)) {
          rest.push_back(tk);
          continue;
        }
        Level& lv = h.levels[tk.l];
        Level& ch = h.levels[tk.l + 1];
        lv.passthru = true;
        lv.k = lv.n;
        lv.t_off.assign(lv.count, 0);
        lv.e_off.assign(lv.count, 0);
        lv.f_off.assign(lv.count, 0);
        lv.g_off.assign(lv.count, 0);
        lv.dh_off.assign(lv.count, 0);
        int64_t dpool = 0;
        std::vector<int> order(lv.ntot);
        for (int j = 0; j < lv.count; ++j) {
          lv.dh_off[j] = dpool;
          dpool += (int64_t)lv.n[j] * lv.n[j];
          for (int i = 0; i < lv.n[j]; ++i) order[lv.off[j] + i] = i;
          h.factor_bytes += 16.0 * lv.n[j] * lv.n[j];
        }
        lv.Dhat.alloc(std::max<int64_t>(dpool, 1));
        lv.perm.upload(order, s);
        for (int j = 0; j < lv.count; ++j)
          dj.push_back({tk.g, lv.idx.get() + lv.off[j], lv.Dhat.get() + lv.dh_off[j], lv.n[j], ch.k[2 * j], 0,
                        ch.Dhat.get() + ch.dh_off[2 * j], ch.Dhat.get() + ch.dh_off[2 * j + 1]});
      }
      if (!dj.empty()) {
        DevBuf<DJob> ddj = upload_jobs(dj, s);
        {
          prof::KScope _ks("k_fill_d", s);
          launch_jobs_y(ddj, dj.size(), [&](const DJob* p, unsigned ny) { k_fill_d<<<dim3(64, ny), 256, 0, s>>>(p); });
        }
        HBS_LAUNCH_CHECK("k_fill_d pass-through");
      }
      tasks.swap(rest);
    }
    if (tasks.empty()) continue;

    // ---- node circles (one stage buffer, one read-back)
    int64_t nodes = 0;
    std::vector<int64_t> node0(tasks.size());
    for (size_t i = 0; i < tasks.size(); ++i) {
      node0[i] = nodes;
      nodes += tasks[i].h->levels[tasks[i].l].count;
    }
    std::vector<double> hcirc;
    {
      DevBuf<double> circ(3 * nodes);
      std::vector<CircleJob> cj;
      for (size_t i = 0; i < tasks.size(); ++i) {
        Handle& h = *tasks[i].h;
        const int l = tasks[i].l;
        const int cnt = 1 << l;
        for (int j = 0; j < cnt; ++j)
          cj.push_back({h.x.get(), h.y.get(), ((int64_t)j * h.N) >> l, ((int64_t)(j + 1) * h.N) >> l,
                        circ.get() + 3 * (node0[i] + j)});
      }
      DevBuf<CircleJob> dcj = upload_jobs(cj, s);
      {
        prof::KScope _ks("k_node_circles", s);
        k_node_circles<<<(unsigned)cj.size(), 128, 0, s>>>(dcj.get());
      }
      HBS_LAUNCH_CHECK("k_node_circles");
      hcirc = circ.download(s);
    }
    for (size_t i = 0; i < tasks.size(); ++i) {
      Level& lv = tasks[i].h->levels[tasks[i].l];
      std::vector<double> cx(lv.count), cy(lv.count);
      lv.h_rad.assign(lv.count, 0.0);
      for (int j = 0; j < lv.count; ++j) {
        cx[j] = hcirc[3 * (node0[i] + j)];
        cy[j] = hcirc[3 * (node0[i] + j) + 1];
        lv.h_rad[j] = hcirc[3 * (node0[i] + j) + 2];
      }
      lv.cx.upload(cx, s);
      lv.cy.upload(cy, s);
      lv.rad.upload(lv.h_rad, s);
    }

    // ---- near lists (count pass, offsets, fill pass)
    std::vector<int64_t> hcnt;
    std::vector<int64_t> noff(nodes, 0);
    DevBuf<int64_t> near;
    {
      DevBuf<int64_t> cnt(nodes);
      // candidate ranges per node: the nodes whose enclosing circle meets its proxy circle,
      // found by a sweep over the centres sorted in x (window: the proxy radius plus the
      // level's largest node radius)
      std::vector<longlong2> hranges;
      std::vector<int64_t> rbeg(nodes + 1, 0);
      for (size_t i = 0; i < tasks.size(); ++i) {
        Level& lv = tasks[i].h->levels[tasks[i].l];
        const double rho = tasks[i].h->opts.proxy_rho;
        const double* hc = hcirc.data() + 3 * node0[i];
        std::vector<int> order(lv.count);
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int a, int b) { return hc[3 * a] < hc[3 * b]; });
        std::vector<double> xs(lv.count);
        double rmax = 0.0;
        for (int q = 0; q < lv.count; ++q) {
          xs[q] = hc[3 * order[q]];
          rmax = std::max(rmax, hc[3 * q + 2]);
        }
        std::vector<int> cand;
        for (int j = 0; j < lv.count; ++j) {
          const double R = rho * lv.h_rad[j];
          // a point of node c lies within r_c of c's centre; the margin covers the rounding
          // of the computed radii
          const double reach = R + rmax * (1.0 + 1e-9) + 1e-12;
          const double cxj = hc[3 * j], cyj = hc[3 * j + 1];
          cand.clear();
          for (auto it = std::lower_bound(xs.begin(), xs.end(), cxj - reach); it != xs.end() && *it <= cxj + reach;
               ++it) {
            const int c = order[it - xs.begin()];
            if (c == j) continue;
            const double lim = R + hc[3 * c + 2] * (1.0 + 1e-9) + 1e-12;
            if (std::hypot(hc[3 * c] - cxj, hc[3 * c + 1] - cyj) < lim) cand.push_back(c);
          }
          std::sort(cand.begin(), cand.end());
          for (int c : cand) {
            const int64_t lo = lv.off[c], hi = lv.off[c] + lv.n[c];
            if (hi <= lo) continue;
            if ((int64_t)hranges.size() > rbeg[node0[i] + j] && hranges.back().y == lo) hranges.back().y = hi;
            else hranges.push_back(make_longlong2(lo, hi));
          }
          rbeg[node0[i] + j + 1] = (int64_t)hranges.size();
        }
      }
      DevBuf<longlong2> dranges;
      dranges.upload(hranges, s);
      std::vector<NearJob> nj;
      for (size_t i = 0; i < tasks.size(); ++i) {
        Handle& h = *tasks[i].h;
        Level& lv = h.levels[tasks[i].l];
        const double rho = h.opts.proxy_rho;
        for (int j = 0; j < lv.count; ++j) {
          const double R = rho * lv.h_rad[j];
          const int64_t q = node0[i] + j;
          nj.push_back({h.x.get(), h.y.get(), lv.idx.get(), dranges.get() + rbeg[q], (int)(rbeg[q + 1] - rbeg[q]),
                        hcirc[3 * q], hcirc[3 * q + 1], R * R, cnt.get() + q, nullptr});
        }
      }
      DevBuf<NearJob> dnj = upload_jobs(nj, s);
      {
        prof::KScope _ks("k_near", s);
        k_near<<<(unsigned)nj.size(), 256, 0, s>>>(dnj.get());
      }
      HBS_LAUNCH_CHECK("k_near count");
      hcnt = cnt.download(s);
      int64_t tot = 0;
      for (int64_t q = 0; q < nodes; ++q) { noff[q] = tot; tot += hcnt[q]; }
      near.alloc(std::max<int64_t>(tot, 1));
      for (int64_t q = 0; q < nodes; ++q) nj[q].out = near.get() + noff[q];
      DevBuf<NearJob> dnj2 = upload_jobs(nj, s);
      {
        prof::KScope _ks("k_near", s);
        k_near<<<(unsigned)nj.size(), 256, 0, s>>>(dnj2.get());
      }
      HBS_LAUNCH_CHECK("k_near fill");
    }

    // ---- ID matrices and the joint IDs (Def. 3.1)
    {
      std::vector<YJob> yj;
      std::vector<int64_t> ymt;
      int64_t ypool = 0;
      for (size_t i = 0; i < tasks.size(); ++i) {
        Handle& h = *tasks[i].h;
        Level& lv = h.levels[tasks[i].l];
        for (int j = 0; j < lv.count; ++j) {
          const double R = h.opts.proxy_rho * lv.h_rad[j];
          // the fastest wavenumber of the operator: w, or n w inside transmission obstacles
          const double kmax = h.comps == 2 ? std::max(h.omega, h.index * h.omega) : h.omega;
          int np = (int)(2.0 * std::ceil(kmax * R) + 40.0);
          np = std::max(np, h.opts.n_proxy_min);
          np = (np + 7) / 8 * 8;
          const int nn = (int)hcnt[node0[i] + j];
          yj.push_back({tasks[i].g, lv.idx.get() + lv.off[j], near.get() + noff[node0[i] + j], nullptr, lv.n[j], nn,
                        np, hcirc[3 * (node0[i] + j)], hcirc[3 * (node0[i] + j) + 1], R, 2.0 * HBS_PI * R / np});
          ymt.push_back(ypool);
          ypool += (int64_t)y_rows(yj.back()) * lv.n[j];
        }
      }
      DevBuf<cplx> Y(std::max<int64_t>(ypool, 1));
      for (size_t q = 0; q < yj.size(); ++q) yj[q].mt = Y.get() + ymt[q];
      DevBuf<YJob> dyj = upload_jobs(yj, s);
      {
        prof::KScope _ks("k_fill_y", s);
        int npmax = 0;
        for (const auto& y : yj) npmax = std::max(npmax, y.np);
        const size_t psm = 4 * (size_t)npmax * sizeof(double);
        bool any1 = false, any2 = false;
        for (const auto& y : yj) (y.g.comps == 2 ? any2 : any1) = true;
        if (psm > 48 * 1024) {
          HBS_CUDA(raise_smem_limit((const void*)k_fill_y, psm));
          HBS_CUDA(raise_smem_limit((const void*)k_fill_y_tr, psm));
        }
        // each kernel skips the jobs of the other problem
        if (any1)
          launch_jobs_y(dyj, yj.size(), [&](const YJob* p, unsigned ny) { k_fill_y<<<dim3(64, ny), 256, psm, s>>>(p); });
        if (any2)
          launch_jobs_y(dyj, yj.size(), [&](const YJob* p, unsigned ny) { k_fill_y_tr<<<dim3(64, ny), 256, psm, s>>>(p); });
      }
      HBS_LAUNCH_CHECK("k_fill_y");
      // The matrix each ID runs on: Mt itself, or on tensor-core handles its randomized
      // sketch when Mt is tall (the published randomized ID: the skeleton and T of the
      // column-pivoted QR of Y = Omega Mt, Omega an l x m matrix of random signs with
      // l = n + 16 rows, approximate those of Mt, whose columns Y's rows sample).  The sketch
      // is one batched product on the tensor cores; the QR then runs on l instead of m rows.
      std::vector<cplx*> idmat(yj.size());
      std::vector<int> idrows(yj.size());
      DevBuf<cplx> Ysk, Om;
      {
        std::vector<GemmJob> sj;
        std::vector<size_t> sq;
        int64_t pool = 0;
        int lmax = 0, mmax = 0;
        for (size_t q = 0; q < yj.size(); ++q) {
          const int m = y_rows(yj[q]), n = yj[q].n;
          idmat[q] = yj[q].mt;
          idrows[q] = m;
          const int l = n + kSketchOver;
          if (!gemm_tensor() || m < 96 || 4 * m < 5 * l) continue;
          sq.push_back(q);
          pool += (int64_t)l * n;
          lmax = std::max(lmax, l);
          mmax = std::max(mmax, m);
        }
        if (!sq.empty()) {
          Om.alloc((size_t)lmax * mmax);
          Ysk.alloc((size_t)pool);
          {
            prof::KScope _ks("k_sketch_signs", s);
            k_sketch_signs<<<grid_1d((int64_t)lmax * mmax), 256, 0, s>>>(Om.get(), lmax, mmax);
          }
          HBS_LAUNCH_CHECK("k_sketch_signs");
          int64_t o = 0;
          for (size_t q : sq) {
            const int m = y_rows(yj[q]), n = yj[q].n, l = n + kSketchOver;
            // Omega's entries are real signs: one digit plane (the tensor-core product skips the rest)
            sj.push_back(GemmJob{Om.get(), yj[q].mt, Ysk.get() + o, l, n, m, lmax, m, l, cmk(1.0, 0.0),
                                 cmk(0.0, 0.0), 0, 0, 0, 0, 0, 1});
            idmat[q] = Ysk.get() + o;
            idrows[q] = l;
            o += (int64_t)l * n;
          }
          run_gemms(sj, s);
        }
      }
      std::vector<CpqrJob> cj;
      for (size_t i = 0; i < tasks.size(); ++i) {
        Level& lv = tasks[i].h->levels[tasks[i].l];
        lv.t_off.assign(lv.count, 0);
        int64_t tpool = 0;
        for (int j = 0; j < lv.count; ++j) {
          const int m = idrows[node0[i] + j];
          lv.t_off[j] = tpool;
          tpool += (int64_t)std::min(m, lv.n[j]) * lv.n[j];
        }
        lv.T.alloc(std::max<int64_t>(tpool, 1));
        lv.perm.alloc(std::max<int64_t>(lv.ntot, 1));
        for (int j = 0; j < lv.count; ++j) {
          const size_t q = node0[i] + j;
          cj.push_back({idmat[q], lv.T.get() + lv.t_off[j], lv.perm.get() + lv.off[j], idrows[q], lv.n[j],
                        (int)cj.size()});
        }
      }
      std::vector<int> ranks = batched_id(cj, tasks[0].h->tol, s);
      for (size_t i = 0; i < tasks.size(); ++i) {
        Handle& h = *tasks[i].h;
        Level& lv = h.levels[tasks[i].l];
        lv.k.assign(ranks.begin() + node0[i], ranks.begin() + node0[i] + lv.count);
        for (int j = 0; j < lv.count; ++j) h.max_rank = std::max(h.max_rank, lv.k[j]);
      }
    }
    near.release();

    // ---- D blocks and their inverses (Dinv becomes G below)
    std::vector<DevBuf<cplx>> Dinv(tasks.size()), X(tasks.size()), Yp(tasks.size()), S(tasks.size());
    std::vector<std::vector<int64_t>> d_off(tasks.size());
    {
      std::vector<DJob> dj;
      std::vector<InvJob> ij;
      for (size_t i = 0; i < tasks.size(); ++i) {
        Handle& h = *tasks[i].h;
        const int l = tasks[i].l;
        Level& lv = h.levels[l];
        d_off[i].assign(lv.count, 0);
        int64_t dpool = 0;
        for (int j = 0; j < lv.count; ++j) { d_off[i][j] = dpool; dpool += (int64_t)lv.n[j] * lv.n[j]; }
        Dinv[i].alloc(std::max<int64_t>(dpool, 1));
        for (int j = 0; j < lv.count; ++j) {
          cplx* d = Dinv[i].get() + d_off[i][j];
          if (l == h.L) {
            dj.push_back({tasks[i].g, lv.idx.get() + lv.off[j], d, lv.n[j], 0, 1, nullptr, nullptr});
          } else {
            Level& ch = h.levels[l + 1];
            dj.push_back({tasks[i].g, lv.idx.get() + lv.off[j], d, lv.n[j], ch.k[2 * j], 0,
                          ch.Dhat.get() + ch.dh_off[2 * j], ch.Dhat.get() + ch.dh_off[2 * j + 1]});
          }
          ij.push_back({d, nullptr, lv.n[j], (int)ij.size()});
        }
      }
      DevBuf<DJob> ddj = upload_jobs(dj, s);
      {
        prof::KScope _ks("k_fill_d", s);
        launch_jobs_y(ddj, dj.size(), [&](const DJob* p, unsigned ny) { k_fill_d<<<dim3(64, ny), 256, 0, s>>>(p); });
      }
      HBS_LAUNCH_CHECK("k_fill_d");
      batched_inverse(ij, s, "leaf/level block");
    }
    // X = D^{-1} P (n x k), Yt = P^T D^{-1} (k x n), S = P^T X (k x k).  With Dp = D^{-1}(:, perm),
    // Dr = D^{-1}(perm, :) and Xr = X(perm, :):
    //   X = Dp(:, :k) + Dp(:, k:) T^T,   Yt = Dr(:k, :) + T Dr(k:, :),   S = Xr(:k, :) + T Xr(k:, :),
    // permuted copies followed by batched GEMMs (double-float or tensor cores).
    {
      std::vector<PermJob> pj1, pj2;
      std::vector<GemmJob> g1, g2;
      std::vector<DevBuf<cplx>> Dp(tasks.size()), Dr(tasks.size()), Xr(tasks.size()), Tt(tasks.size());
      for (size_t i = 0; i < tasks.size(); ++i) {
        Level& lv = tasks[i].h->levels[tasks[i].l];
        lv.e_off.assign(lv.count, 0); lv.f_off.assign(lv.count, 0); lv.dh_off.assign(lv.count, 0);
        int64_t eo = 0, dho = 0, nno = 0, tto = 0;
        std::vector<int64_t> nn_off(lv.count), tt_off(lv.count);
        for (int j = 0; j < lv.count; ++j) {
          lv.e_off[j] = eo; lv.f_off[j] = eo; eo += (int64_t)lv.n[j] * lv.k[j];
          lv.dh_off[j] = dho; dho += (int64_t)lv.k[j] * lv.k[j];
          nn_off[j] = nno; nno += (int64_t)lv.n[j] * lv.n[j];
          tt_off[j] = tto; tto += (int64_t)(lv.n[j] - lv.k[j]) * lv.k[j];
        }
        X[i].alloc(std::max<int64_t>(eo, 1));
        Yp[i].alloc(std::max<int64_t>(eo, 1));
        S[i].alloc(std::max<int64_t>(dho, 1));
        Dp[i].alloc(std::max<int64_t>(nno, 1));
        Dr[i].alloc(std::max<int64_t>(nno, 1));
        Xr[i].alloc(std::max<int64_t>(eo, 1));
        Tt[i].alloc(std::max<int64_t>(tto, 1));
        for (int j = 0; j < lv.count; ++j) {
          const int n = lv.n[j], k = lv.k[j], nk = n - k;
          if (k == 0) continue;
          const int* pm = lv.perm.get() + lv.off[j];
          const cplx* T = lv.T.get() + lv.t_off[j];
          const cplx* d = Dinv[i].get() + d_off[i][j];
          cplx* dp = Dp[i].get() + nn_off[j];
          cplx* dr = Dr[i].get() + nn_off[j];
          cplx* x = X[i].get() + lv.e_off[j];
          cplx* yt = Yp[i].get() + lv.f_off[j];
          cplx* xr = Xr[i].get() + lv.e_off[j];
          cplx* tt = Tt[i].get() + tt_off[j];
          pj1.push_back({d, dp, x, pm, T, nk > 0 ? tt : nullptr, n, k, n, n, 0});
          pj1.push_back({d, dr, yt, pm, nullptr, nullptr, n, k, n, n, 1});
          pj2.push_back({x, xr, S[i].get() + lv.dh_off[j], pm, nullptr, nullptr, n, k, k, n, 1});
          if (nk > 0) {
            // X += Dp(:, k:) Tt   (n x nk) (nk x k)
            g1.push_back({dp + (int64_t)k * n, tt, x, n, k, nk, n, nk, n, cmk(1, 0), cmk(1, 0), 0, 0, 0});
            // Yt += T Dr(k:, :)    (k x nk) (nk x n)
            g1.push_back({T, dr + k, yt, k, n, nk, k, n, k, cmk(1, 0), cmk(1, 0), 0, 0, 0});
            // S += T Xr(k:, :)     (k x nk) (nk x k)
            g2.push_back({T, xr + k, S[i].get() + lv.dh_off[j], k, k, nk, k, n, k, cmk(1, 0), cmk(1, 0), 0, 0, 0});
          }
        }
      }
      {
        DevBuf<PermJob> dp1 = upload_jobs(pj1, s);
        prof::KScope _ks("k_perm_copy", s);
        launch_jobs_y(dp1, pj1.size(), [&](const PermJob* p, unsigned ny) { k_perm_copy<<<dim3(32, ny), 256, 0, s>>>(p); });
      }
      HBS_LAUNCH_CHECK("k_perm_copy");
      launch_gemms(g1, s);
      {
        DevBuf<PermJob> dp2 = upload_jobs(pj2, s);
        prof::KScope _ks("k_perm_copy", s);
        launch_jobs_y(dp2, pj2.size(), [&](const PermJob* p, unsigned ny) { k_perm_copy<<<dim3(32, ny), 256, 0, s>>>(p); });
      }
      HBS_LAUNCH_CHECK("k_perm_copy X");
      launch_gemms(g2, s);
      HBS_CUDA(cudaStreamSynchronize(s));
    }
    // Dhat = S^{-1}
    {
      std::vector<InvJob> ij;
      for (size_t i = 0; i < tasks.size(); ++i) {
        Level& lv = tasks[i].h->levels[tasks[i].l];
        for (int j = 0; j < lv.count; ++j)
          if (lv.k[j] > 0) ij.push_back({S[i].get() + lv.dh_off[j], nullptr, lv.k[j], (int)ij.size()});
      }
      batched_inverse(ij, s, "skeleton block P^T D^-1 P");
    }
    // E = X Dhat, F* = Dhat Yt, G = D^{-1} - E Yt
    {
      std::vector<GemmJob> g1, g2;
      for (size_t i = 0; i < tasks.size(); ++i) {
        Handle& h = *tasks[i].h;
        Level& lv = h.levels[tasks[i].l];
        int64_t eo = 0;
        for (int j = 0; j < lv.count; ++j) eo += (int64_t)lv.n[j] * lv.k[j];
        lv.Dhat = std::move(S[i]);
        lv.E.alloc(std::max<int64_t>(eo, 1));
        lv.F.alloc(std::max<int64_t>(eo, 1));
        lv.G = std::move(Dinv[i]);
        lv.g_off = d_off[i];
        for (int j = 0; j < lv.count; ++j) {
          const int n = lv.n[j], k = lv.k[j];
          if (k == 0) continue;
          g1.push_back({X[i].get() + lv.e_off[j], lv.Dhat.get() + lv.dh_off[j], lv.E.get() + lv.e_off[j], n, k, k, n,
                        k, n, cmk(1, 0), cmk(0, 0), 0, 0, 0});
          g1.push_back({lv.Dhat.get() + lv.dh_off[j], Yp[i].get() + lv.f_off[j], lv.F.get() + lv.f_off[j], k, n, k, k,
                        k, k, cmk(1, 0), cmk(0, 0), 0, 0, 0});
          g2.push_back({lv.E.get() + lv.e_off[j], Yp[i].get() + lv.f_off[j], lv.G.get() + lv.g_off[j], n, n, k, n, k,
                        n, cmk(-1, 0), cmk(1, 0), 0, 0, 0});
        }
        for (int j = 0; j < lv.count; ++j) {
          const double n = lv.n[j], k = lv.k[j];
          h.factor_bytes += 16.0 * (2 * n * k + n * n);
          h.apply_flops += 8.0 * (2 * n * k + n * n);
        }
      }
      launch_gemms(g1, s);
      launch_gemms(g2, s);
    }
  }
}

void build_hbs(Handle& h, cudaStream_t s) {
  std::vector<Handle*> one{&h};
  build_hbs_multi(one, s);
}

// x = A^{-1} b through the telescoping factorization (Sec. 4): upward b^_tau = F*_tau b_tau,
// root solve, downward x_tau = E_tau x^_tau + G_tau b_tau.
// x = A^{-1} b (trans = false) or x = A^{-T} b (trans = true, the factors transposed:
// A^{-T} = F*^T (M~ + Dhat)^{-T} E^T + G^T, applied with the same telescoping sweep).
// Y = Op^T X for a factor Op (stored rows x cols, ld) and a level vector X (rows x nrhs):
// formed as Y^T = X^T Op (nrhs x cols, Y written row-major), so that the many right-hand
// sides fill the 128-row tiles of the tensor-core products even at the leaves.
static void tprod(std::vector<GemmJob>& gj, int64_t nrhs, const cplx* Op, int rows, int cols, int ld, const cplx* X,
                  int64_t ldx, cplx* Y, int64_t ldy, cplx beta) {
  GemmJob j{};
  j.A = X;
  j.lda = (int)ldx;
  j.transA = 1;
  j.B = Op;
  j.ldb = ld;
  j.C = Y;
  j.ldc = (int)ldy;
  j.transC = 1;
  j.m = (int)nrhs;
  j.n = cols;
  j.k = rows;
  j.alpha = cmk(1, 0);
  j.beta = beta;
  gj.push_back(j);
}

// The upward step of level l (1 <= l <= L): up[l - 1] = F* b_tau (or E^T b_tau) for every
// node, from level l's vector (b itself at the leaves).  The parent level's offsets follow
// from level l's ranks (a parent's size is the sum of its two children's ranks).
static void sweep_upward_level(const Handle& H, int l, const cplx* b, int64_t nrhs, bool trans,
                        std::vector<DevBuf<cplx>>& up, cudaStream_t s) {
  const Level& lv = H.levels[l];
  const int np = lv.count / 2;
  std::vector<int64_t> poff(std::max(np, 1), 0);
  int64_t pnt = 0;
  for (int p = 0; p < np; ++p) {
    poff[p] = pnt;
    pnt += lv.k[2 * p] + lv.k[2 * p + 1];
  }
  if ((int)up.size() < H.L + 1) up.resize(H.L + 1);
  up[l - 1].alloc(std::max<int64_t>(pnt * nrhs, 1));
  const cplx* in = l == H.L ? b : up[l].get();
  if (lv.passthru) {  // F* = E^T = I: the parent's vector is this level's (same layout, pnt = ntot)
    if (pnt * nrhs > 0)
      HBS_CUDA(cudaMemcpyAsync(up[l - 1].get(), in, sizeof(cplx) * pnt * nrhs, cudaMemcpyDeviceToDevice, s));
    return;
  }
  std::vector<GemmJob> gj;
  for (int j = 0; j < lv.count; ++j) {
    const int n = lv.n[j], k = lv.k[j];
    if (k == 0) continue;
    const int64_t prow = poff[j >> 1] + ((j & 1) ? lv.k[j - 1] : 0);
    if (trans)  // E^T b (E stored n x k)
      tprod(gj, nrhs, lv.E.get() + lv.e_off[j], n, k, n, in + lv.off[j], lv.ntot, up[l - 1].get() + prow, pnt,
            cmk(0, 0));
    else  // F* b (F* stored k x n)
      gj.push_back({lv.F.get() + lv.f_off[j], in + lv.off[j], up[l - 1].get() + prow, k, (int)nrhs, n, k,
                    (int)lv.ntot, (int)pnt, cmk(1, 0), cmk(0, 0), 0, 0, 0, 0, 0});
  }
  run_gemms(gj, s);
}

// The rest of the sweep once every upward step is done: the root solve and the downward
// steps, x_tau = G b_tau + E x^_tau (or G^T b_tau + F*^T x^_tau).
static void sweep_finish(const Handle& H, const cplx* b, cplx* xout, int64_t nrhs, bool trans,
                  std::vector<DevBuf<cplx>>& up, cudaStream_t s) {
  const int Lv = H.L;
  const auto& levels = H.levels;
  std::vector<DevBuf<cplx>> dn(Lv + 1);
  for (int l = 0; l < Lv; ++l) dn[l].alloc(std::max<int64_t>(levels[l].ntot * nrhs, 1));
  auto upptr = [&](int l) -> const cplx* { return l == Lv ? b : up[l].get(); };
  {
    std::vector<GemmJob> gj;
    if (trans)
      tprod(gj, nrhs, H.Groot.get(), H.nroot, H.nroot, H.nroot, up[0].get(), H.nroot, dn[0].get(), H.nroot, cmk(0, 0));
    else
      gj.push_back({H.Groot.get(), up[0].get(), dn[0].get(), H.nroot, (int)nrhs, H.nroot, H.nroot, H.nroot, H.nroot,
                    cmk(1, 0), cmk(0, 0), 0, 0, 0, 0, 0});
    run_gemms(gj, s);
  }
  for (int l = 1; l <= Lv; ++l) {
    const Level& lv = levels[l];
    const Level& pa = levels[l - 1];
    cplx* outp = l == Lv ? xout : dn[l].get();
    if (lv.passthru) {  // G = 0, E = F*^T = I: x_tau = x^_tau (same layout)
      if (lv.ntot * nrhs > 0)
        HBS_CUDA(cudaMemcpyAsync(outp, dn[l - 1].get(), sizeof(cplx) * lv.ntot * nrhs, cudaMemcpyDeviceToDevice, s));
      continue;
    }
    std::vector<GemmJob> gj;
    for (int j = 0; j < lv.count; ++j) {
      const int n = lv.n[j];
      // x_tau = G b_tau  (or G^T b_tau)
      if (trans)
        tprod(gj, nrhs, lv.G.get() + lv.g_off[j], n, n, n, upptr(l) + lv.off[j], lv.ntot, outp + lv.off[j], lv.ntot,
              cmk(0, 0));
      else
        gj.push_back({lv.G.get() + lv.g_off[j], upptr(l) + lv.off[j], outp + lv.off[j], n, (int)nrhs, n, n,
                      (int)lv.ntot, (int)lv.ntot, cmk(1, 0), cmk(0, 0), 0, 0, 0, 0, 0});
    }
    run_gemms(gj, s);
    gj.clear();
    for (int j = 0; j < lv.count; ++j) {
      const int n = lv.n[j], k = lv.k[j];
      if (k == 0) continue;
      const int parent = j >> 1;
      const int64_t prow = pa.off[parent] + ((j & 1) ? levels[l].k[j - 1] : 0);
      if (trans) {
        // x_tau += F*^T x^_tau  (F* stored k x n)
        tprod(gj, nrhs, lv.F.get() + lv.f_off[j], k, n, k, dn[l - 1].get() + prow, pa.ntot, outp + lv.off[j],
              lv.ntot, cmk(1, 0));
      } else {
        // x_tau += E x^_tau  (E stored n x k)
        gj.push_back({lv.E.get() + lv.e_off[j], dn[l - 1].get() + prow, outp + lv.off[j], n, (int)nrhs, k, n,
                      (int)pa.ntot, (int)lv.ntot, cmk(1, 0), cmk(1, 0), 0, 0, 0, 0, 0});
      }
    }
    run_gemms(gj, s);
  }
}

static void apply_impl(const Handle& H, const cplx* b, cplx* xout, int64_t nrhs, cudaStream_t s, bool trans) {
  if (nrhs <= 0) return;
  std::vector<DevBuf<cplx>> up(H.L + 1);
  for (int l = H.L; l >= 1; --l) sweep_upward_level(H, l, b, nrhs, trans, up, s);
  sweep_finish(H, b, xout, nrhs, trans, up, s);
}

void Handle::apply_inverse(const cplx* b, cplx* xout, int64_t nrhs, cudaStream_t s) const {
  apply_impl(*this, b, xout, nrhs, s, false);
}

void Handle::apply_inverse_transpose(const cplx* b, cplx* xout, int64_t nrhs, cudaStream_t s) const {
  apply_impl(*this, b, xout, nrhs, s, true);
}

}  // namespace hbs
