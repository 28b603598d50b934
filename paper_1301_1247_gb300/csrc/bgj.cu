// Blocked Gauss-Jordan inversion with partial pivoting for the large per-node blocks of the
// HBS inversion (the D_tau of Eqs. def_muhD..def_muG at the top tree levels).
//
// Step c of Gauss-Jordan with pivot row r and pivot p = A(r, c) scales row r by 1/p,
// subtracts col_i / p times it from every other row i (col = A(:, c) before the step), and
// stores -col_i / p and 1/p in column c.  Rows are never swapped: r is the largest remaining
// entry of the current column among the rows not yet used as pivots (lowest index on ties),
// and the result X of all n steps is a permutation of the inverse,
// A^{-1}(i, j) = X(pi(i), pi^{-1}(j)) with pi(c) = r.
//
// The steps are taken in panels of b columns (k_bgj_panel: one cluster of CTAs per block,
// the panel in their shared memory).  Within a panel
//   * the panel's own b columns are kept current and updated step by step, as in the
//     unblocked algorithm;
//   * every other column j is left alone; step t records u_t = col (0 in the pivot row) and
//     v_t(j) = (current row r_t)(j) / p_t, the current row coming from
//     row = A(r_t, :) - U(r_t, 0:t) V(:, 0:t)^T.
// At the end of the panel the other columns take the rank-b update A <- A - U V^T in the
// library's batched GEMM (double-float or tensor cores on handles built that way), so the
// O(n^3) work runs as products instead of n dependent column sweeps.  The b pivot rows are
// then set from their own recurrence, X(r_t, j) = v_t(j) - sum_{t' > t} u_{t'}(r_t) v_{t'}(j):
// written as a rank-b update they would cancel (the pivot row scaled in place by 1/p is
// A(r, j) - (1 - 1/p) A(r, j)), costing a factor |p| of accuracy.
#include <algorithm>

#include <cooperative_groups.h>

#include "dense_kernels.cuh"
#include "profile.hpp"
#include "qp_kernels.cuh"
#include "zgemm.cuh"

namespace hbs {

namespace {

constexpr int kCNT = 256;     // threads per CTA of the panel kernel
constexpr const char* kBgjUnavailable = "blocked Gauss-Jordan launch shape unavailable";
constexpr int kMaxPanel = 32;
// shared memory one CTA may use for its slice of the panel (P, U and V rows, used flags)
constexpr size_t kSmemBudget = 200 * 1024;

struct BgjJob {
  cplx* A;        // n x n, ld n, inverted in place
  int n;
  int* pi;        // pivot row of each column
  int* used;      // 1 for rows already used as pivots (zeroed before the first panel)
  cplx* U;        // n x b, ld n
  cplx* V;        // n x b, ld n
  cplx* Vt;       // b x n, ld b (V^T, the GEMM's second operand)
  cplx* tmp;      // n x n scratch for the final permutation
  int* singular;
};

// A CTA's pivot candidate of one step, read by the other CTAs of the cluster: its key and
// row, and that row's entries in the panel's columns and in U.
struct PanelSlot {
  long long key;
  int row;
  int pad;
  cplx prow[kMaxPanel];
  cplx urow[kMaxPanel];
};

// Steps c0 .. c0 + b - 1 of one matrix per cluster of CS CTAs.  CTA q of the cluster owns
// rows [lo, hi) and the same range of columns, with R = ceil(n / CS): its rows of the
// panel's columns (P), of U and its columns' V entries stay in its shared memory.  A step:
//   1. each CTA proposes its largest unused entry of the current pivot column and
//      publishes that row's P and U entries in its slot (slots alternate by step parity);
//   2. one cluster barrier; every CTA reads the CS proposals through distributed shared
//      memory and takes the same winner r (largest key, lowest row on ties), whose P and U
//      rows it copies from the winner's slot;
//   3. each CTA applies the elimination to its rows of the panel and records u_t (its rows)
//      and v_t (its columns outside the panel: the current row r from
//      A(r, j) - U(r, 0:t) V(j, 0:t)^T, scaled by 1/p).
// The loop bounds are the same in every CTA of a cluster, so all of them meet every barrier.
template <int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(kCNT) k_bgj_panel(const BgjJob* jobs, int c0, int b) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ cplx s_dyn[];
  __shared__ PanelSlot slot[2];
  __shared__ cplx s_prow[kMaxPanel], s_pr[kMaxPanel], s_urow[kMaxPanel];
  __shared__ long long redv[kCNT / 32];
  __shared__ int redi[kCNT / 32];
  __shared__ int s_r, s_win;
  __shared__ long long s_key;
  const int q = (int)cluster.block_rank();
  const BgjJob jb = jobs[blockIdx.x / CS];
  const int n = jb.n;
  if (c0 >= n) return;  // the same decision in every CTA of the cluster
  const int bb = min(b, n - c0);
  const int R = (n + CS - 1) / CS;
  const int lo = min(n, q * R), hi = min(n, lo + R), nr = hi - lo;
  const int tid = threadIdx.x;
  cplx* P = s_dyn;           // R x b: P(i - lo, tt) = current A(i, c0 + tt)
  cplx* Uo = P + R * b;      // R x b: U of the own rows
  cplx* Vo = Uo + R * b;     // R x b: V of the own columns
  int* used = reinterpret_cast<int*>(Vo + R * b);
  const cplx* A = jb.A;
  for (int e = tid; e < nr * bb; e += kCNT) {
    const int il = e % nr, tt = e / nr;
    P[il + tt * R] = A[(int64_t)(c0 + tt) * n + lo + il];
  }
  for (int il = tid; il < nr; il += kCNT) used[il] = jb.used[lo + il];
  __syncthreads();
  for (int t = 0; t < bb; ++t) {
    const int c = c0 + t, par = t & 1;
    // 1. this CTA's candidate
    long long best = kNoKey;
    int bi = 0x7fffffff;
    for (int il = tid; il < nr; il += kCNT) {
      if (used[il]) continue;
      const long long key = nkey(cabs2(P[il + t * R]));
      if (better(key, lo + il, best, bi)) { best = key; bi = lo + il; }
    }
    long long bv;
    int br;
    block_argmax_key<kCNT>(best, bi, redv, redi, &bv, &br);  // synchronizes the block
    PanelSlot& my = slot[par];
    if (tid == 0) { my.key = bv; my.row = br; }
    if (br >= lo && br < hi) {
      if (tid < bb) my.prow[tid] = P[(br - lo) + tid * R];
      if (tid < t) my.urow[tid] = Uo[(br - lo) + tid * R];
    }
    cluster.sync();
    // 2. the winner over the cluster, the same in every CTA
    if (tid < 32) {
      long long k2 = kNoKey;
      int r2 = 0x7fffffff, w2 = 0;
      if (tid < CS) {
        const PanelSlot* rs = cluster.map_shared_rank(&slot[par], tid);
        k2 = rs->key;
        r2 = rs->row;
        w2 = tid;
      }
      for (int o = 16; o > 0; o >>= 1) {
        const long long ko = __shfl_xor_sync(0xffffffffu, k2, o);
        const int ro = __shfl_xor_sync(0xffffffffu, r2, o);
        const int wo = __shfl_xor_sync(0xffffffffu, w2, o);
        if (better(ko, ro, k2, r2)) { k2 = ko; r2 = ro; w2 = wo; }
      }
      if (tid == 0) { s_key = k2; s_r = r2; s_win = w2; }
    }
    __syncthreads();
    const long long wkey = s_key;
    int r = s_r;
    const bool nonzero = __longlong_as_double(wkey) > 0.0;
    const bool valid = r >= 0 && r < n;
    if (valid) {
      const PanelSlot* ws = cluster.map_shared_rank(&slot[par], s_win);
      if (tid < bb) s_prow[tid] = ws->prow[tid];
      if (tid < t) s_urow[tid] = ws->urow[tid];
    } else {
      r = c;  // no unused row left cannot happen before step n; keeps indices in range
      if (tid < bb) s_prow[tid] = cmk(0.0, 0.0);
      if (tid < t) s_urow[tid] = cmk(0.0, 0.0);
    }
    __syncthreads();
    const cplx p = s_prow[t];
    const cplx ip = nonzero ? cdiv(cmk(1.0, 0.0), p) : cmk(0.0, 0.0);
    if (tid < bb) s_pr[tid] = cmul(s_prow[tid], ip);
    if (tid == 0) {
      if (q == 0) {
        jb.pi[c] = r;
        if (!nonzero) *jb.singular = 1;
      }
      if (r >= lo && r < hi) used[r - lo] = 1;
    }
    __syncthreads();
    // 3. own rows of the panel and of u_t
    for (int il = tid; il < nr; il += kCNT) {
      const int i = lo + il;
      const cplx col = P[il + t * R];
      cplx u;
      if (i == r) {
        for (int tt = 0; tt < bb; ++tt) P[il + tt * R] = (tt == t) ? ip : s_pr[tt];
        u = cmk(0.0, 0.0);
      } else {
        for (int tt = 0; tt < bb; ++tt) {
          if (tt == t) continue;
          P[il + tt * R] = cfms(col, s_pr[tt], P[il + tt * R]);
        }
        const cplx x = cmul(col, ip);
        P[il + t * R] = cmk(-x.x, -x.y);
        u = col;
      }
      Uo[il + t * R] = u;
      jb.U[(int64_t)t * n + i] = u;
    }
    // own columns outside the panel: v_t
    for (int jl = tid; jl < nr; jl += kCNT) {
      const int j = lo + jl;
      cplx v = cmk(0.0, 0.0);
      if (j < c0 || j >= c0 + bb) {
        cplx acc = A[(int64_t)j * n + r];
#pragma unroll 8
        for (int s2 = 0; s2 < t; ++s2) acc = cfms(s_urow[s2], Vo[jl + s2 * R], acc);
        v = cmul(acc, ip);
      }
      Vo[jl + t * R] = v;
      jb.V[(int64_t)t * n + j] = v;
      jb.Vt[(int64_t)j * b + t] = v;
    }
    __syncthreads();  // P, U, V and the used flags before the next step's proposal
  }
  // the panel's final columns and the used flags of the own rows
  for (int e = tid; e < nr * bb; e += kCNT) {
    const int il = e % nr, tt = e / nr;
    jb.A[(int64_t)(c0 + tt) * n + lo + il] = P[il + tt * R];
  }
  for (int il = tid; il < nr; il += kCNT) jb.used[lo + il] = used[il];
  cluster.sync();  // no CTA leaves while another may still read its slots
}

// After the GEMM: the pivot rows r_t of the columns outside the panel, from
// X(r_t, j) = v_t(j) - sum_{t' > t} u_{t'}(r_t) v_{t'}(j).  Block (32, 8): x runs over 32
// columns, y over the steps t; the b x b coefficients u_{t'}(r_t) are staged in shared memory.
__global__ void __launch_bounds__(256) k_bgj_rows(const BgjJob* jobs, int c0, int b) {
  __shared__ cplx s_u[kMaxPanel * kMaxPanel];  // s_u[t * b + t2] = U(r_t, t2)
  const BgjJob jb = jobs[blockIdx.y];
  const int n = jb.n;
  if (c0 >= n) return;
  const int bb = min(b, n - c0);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int e = tid; e < bb * bb; e += 256) {
    const int t = e / bb, t2 = e % bb;
    s_u[t * bb + t2] = jb.U[(int64_t)t2 * n + jb.pi[c0 + t]];
  }
  __syncthreads();
  for (int j = blockIdx.x * 32 + threadIdx.x; j < n; j += gridDim.x * 32) {
    if (j >= c0 && j < c0 + bb) continue;
    for (int t = threadIdx.y; t < bb; t += 8) {
      cplx acc = jb.V[(int64_t)t * n + j];
#pragma unroll 8
      for (int t2 = t + 1; t2 < bb; ++t2) acc = cfms(s_u[t * bb + t2], jb.V[(int64_t)t2 * n + j], acc);
      jb.A[(int64_t)j * n + jb.pi[c0 + t]] = acc;
    }
  }
}

// tmp(i, j) = X(pi(i), pi^{-1}(j)), then copied back by k_bgj_copy.
__global__ void __launch_bounds__(256) k_bgj_unpermute(const BgjJob* jobs) {
  extern __shared__ int pinv[];
  const BgjJob jb = jobs[blockIdx.y];
  const int n = jb.n;
  for (int c = threadIdx.x; c < n; c += blockDim.x) pinv[jb.pi[c]] = c;
  __syncthreads();
  const int64_t tot = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    jb.tmp[e] = jb.A[(int64_t)pinv[j] * n + jb.pi[i]];
  }
}

__global__ void k_bgj_copy(const BgjJob* jobs) {
  const BgjJob jb = jobs[blockIdx.y];
  const int64_t tot = (int64_t)jb.n * jb.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
    jb.A[e] = jb.tmp[e];
}

}  // namespace

static size_t bgj_slice_bytes(int R, int b) { return (size_t)R * b * 3 * sizeof(cplx) + (size_t)R * sizeof(int); }

// Panel width for blocks up to nmax on clusters of cs CTAs (0: does not fit).
bool bgj_unavailable(const Error& e) { return std::string(e.what()).rfind(kBgjUnavailable, 0) == 0; }

int bgj_panel_width(int nmax, int cs) {
  const int R = (nmax + cs - 1) / cs;
  int b = kMaxPanel;
  while (b > 8 && bgj_slice_bytes(R, b) > kSmemBudget) b /= 2;
  return bgj_slice_bytes(R, b) <= kSmemBudget ? b : 0;
}

template <int CS>
static void launch_bgj_panel(const BgjJob* dj, int nj, int c0, int b, size_t smem, cudaStream_t s) {
  HBS_CUDA(raise_smem_limit((const void*)k_bgj_panel<CS>, smem));
  k_bgj_panel<CS><<<(unsigned)(nj * CS), kCNT, smem, s>>>(dj, c0, b);
}

// Clusters of this launch shape the device can hold at once (0: it cannot run one).
template <int CS>
static int bgj_max_clusters(size_t smem) {
  if (raise_smem_limit((const void*)k_bgj_panel<CS>, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(CS, 1, 1);
  cfg.blockDim = dim3(kCNT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_bgj_panel<CS>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

void bgj_run(const std::vector<std::pair<cplx*, int>>& mats, int cs, cudaStream_t s, const char* what) {
  const int nj = (int)mats.size();
  if (nj == 0) return;
  int nmax = 0;
  int64_t ntot = 0, atot = 0;
  for (const auto& m : mats) {
    if (m.second < 1) throw Error(HBS_ERR_INTERNAL, "blocked Gauss-Jordan: empty block");
    nmax = std::max(nmax, m.second);
    ntot += m.second;
    atot += (int64_t)m.second * m.second;
  }
  // cluster size cs (1, 2, 4 or 8 CTAs per block, each with a slice of R = ceil(n / cs)
  // rows); panel width: the widest of 32, 16, 8 whose slice fits in shared memory
  if (cs != 1 && cs != 2 && cs != 4 && cs != 8) throw Error(HBS_ERR_INTERNAL, "blocked Gauss-Jordan: cluster size");
  const int CS = cs;
  const int b = bgj_panel_width(nmax, CS);
  if (b == 0) throw Error(HBS_ERR_INVALID_ARG, "blocked Gauss-Jordan: block too large for the cluster");
  const int R = (nmax + CS - 1) / CS;
  const size_t smem = bgj_slice_bytes(R, b);
  int fits = 0;
  switch (CS) {
    case 8: fits = bgj_max_clusters<8>(smem); break;
    case 4: fits = bgj_max_clusters<4>(smem); break;
    case 2: fits = bgj_max_clusters<2>(smem); break;
    default: fits = bgj_max_clusters<1>(smem); break;
  }
  if (fits < 1) throw Error(HBS_ERR_INTERNAL, std::string(kBgjUnavailable) + ": no cluster of this shape fits");
  DevBuf<int> pi(ntot), used(ntot), sing(nj);
  DevBuf<cplx> U(ntot * b), V(ntot * b), Vt(ntot * b), tmp(atot);
  HBS_CUDA(cudaMemsetAsync(used.get(), 0, sizeof(int) * ntot, s));
  HBS_CUDA(cudaMemsetAsync(sing.get(), 0, sizeof(int) * nj, s));
  std::vector<BgjJob> jobs(nj);
  int64_t o = 0, ao = 0;
  for (int j = 0; j < nj; ++j) {
    const int n = mats[j].second;
    jobs[j] = {mats[j].first, n, pi.get() + o, used.get() + o, U.get() + o * b, V.get() + o * b, Vt.get() + o * b,
               tmp.get() + ao, sing.get() + j};
    o += n;
    ao += (int64_t)n * n;
  }
  DevBuf<BgjJob> dj;
  dj.upload(jobs, s);
  // the panels' own work (per step: the current pivot row, n t, and the panel's columns,
  // n b complex multiply-adds); the rank-b updates are counted by the GEMM kernels
  double fl = 0.0;
  for (const auto& m : mats)
    for (int c0 = 0; c0 < m.second; c0 += b) {
      const double bb = std::min(b, m.second - c0);
      fl += 8.0 * m.second * bb * (1.5 * bb);
    }
  for (int c0 = 0; c0 < nmax; c0 += b) {
    {
      prof::KScope _ks("k_bgj_panel", s);
      switch (CS) {
        case 8: launch_bgj_panel<8>(dj.get(), nj, c0, b, smem, s); break;
        case 4: launch_bgj_panel<4>(dj.get(), nj, c0, b, smem, s); break;
        case 2: launch_bgj_panel<2>(dj.get(), nj, c0, b, smem, s); break;
        default: launch_bgj_panel<1>(dj.get(), nj, c0, b, smem, s); break;
      }
    }
    if (c0 == 0) {
      // a launch the device rejects never ran: the blocks are untouched, the caller may fall back
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess)
        throw Error(HBS_ERR_INTERNAL, std::string(kBgjUnavailable) + ": " + cudaGetErrorString(e));
    }
    HBS_LAUNCH_CHECK("k_bgj_panel");
    // A <- A - U V^T on the columns outside the panel (left and right of it)
    std::vector<GemmJob> g;
    for (const auto& jb : jobs) {
      if (jb.n <= c0) continue;
      const int bb = std::min(b, jb.n - c0);
      const int parts[2][2] = {{0, c0}, {c0 + bb, jb.n - c0 - bb}};
      for (const auto& pt : parts) {
        if (pt[1] <= 0) continue;
        GemmJob gj{};
        gj.A = jb.U;
        gj.B = jb.Vt + (int64_t)pt[0] * b;
        gj.C = jb.A + (int64_t)pt[0] * jb.n;
        gj.m = jb.n;
        gj.n = pt[1];
        gj.k = bb;
        gj.lda = jb.n;
        gj.ldb = b;
        gj.ldc = jb.n;
        gj.alpha = cmk(-1.0, 0.0);
        gj.beta = cmk(1.0, 0.0);
        g.push_back(gj);
      }
    }
    run_gemms(g, s);
    {
      prof::KScope _ks("k_bgj_rows", s);
      k_bgj_rows<<<dim3((unsigned)std::min(64, (nmax + 31) / 32), nj), dim3(32, 8), 0, s>>>(dj.get(), c0, b);
    }
    HBS_LAUNCH_CHECK("k_bgj_rows");
  }
  {
    prof::KScope _ks("k_bgj_unpermute", s);
    const unsigned bx = (unsigned)std::max(1, 1216 / nj);
    const size_t sm = (size_t)nmax * sizeof(int);
    HBS_CUDA(raise_smem_limit((const void*)k_bgj_unpermute, sm));
    k_bgj_unpermute<<<dim3(bx, nj), 256, sm, s>>>(dj.get());
    k_bgj_copy<<<dim3(bx, nj), 256, 0, s>>>(dj.get());
  }
  HBS_LAUNCH_CHECK("k_bgj_unpermute");
  prof::add_work("k_bgj_panel", fl, 0.0);
  auto hsg = sing.download(s);
  for (int j = 0; j < nj; ++j)
    if (hsg[j]) throw Error(HBS_WARN_ILLCOND, std::string("singular block in ") + what);
}

}  // namespace hbs
