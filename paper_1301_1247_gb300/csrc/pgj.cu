// Persistent Gauss-Jordan inversion with partial pivoting for the large per-node blocks
// of the HBS inversion (the D_tau of Eqs. def_muhD..def_muG at the top tree levels).
// One cooperative launch runs every column step of every matrix in a batch, with one
// barrier per step among the CTAs of each matrix.
//
// Step c of a matrix: every CTA of the matrix copies column c into shared memory and takes
// the pivot row p (largest modulus among rows >= c, lowest index on ties) and 1/pivot from
// the slot that the owner of column c filled right after updating it in step c - 1 (so no
// CTA searches or divides on the critical path between two barriers).  Each warp owns a
// fixed set of columns j != c and applies the row interchange (c, p), the scaling of row c
// and the elimination to them.  Column c itself must stay untouched until every CTA has
// read it, so its owner writes its final values (1/pivot in row c, -A(i,c)/pivot
// elsewhere) at the start of step c+1, from the copy kept in shared memory, before
// applying step c+1 to it.  The row interchanges are undone at the end as one column
// permutation (k_pgj_unpivot).
#include <algorithm>

#include "dense_kernels.cuh"
#include "dfloat.cuh"
#include "gridsync.cuh"
#include "profile.hpp"
#include "qp_kernels.cuh"

namespace hbs {

namespace {

constexpr int kNT = 256;
constexpr int kNW = kNT / 32;

struct PgjJob {
  cplx* A;   // n x n, ld n, inverted in place
  int n;
  int b0, nb;
  int* piv;  // n
  int* singular;
  cplx* tmp;  // n x n scratch for the final column permutation
  // pivot of the next step (parity slots), found by the owner of that column right after
  // updating it: row, nonzero flag, and the reciprocal of the pivot (dfc bits in DF mode)
  int* la_p;
  int* la_nz;
  cplx* la_ip;
  GridSync* gs;  // barrier of this matrix's CTAs
};

// The next pivot of column `col` (rows >= c) by its owning warp, from its current values:
// lowest row of largest modulus (keys as in the block search), written to slot c & 1.
template <bool DF>
__device__ __forceinline__ void pgj_lookahead(const PgjJob& jb, const cplx* colp, int c, int lane) {
  const int n = jb.n;
  long long best = kNoKey;
  int bi = 0x7fffffff;
  for (int i = c + lane; i < n; i += 32) {
    long long a;
    if constexpr (DF) {
      const dfc v = reinterpret_cast<const dfc*>(colp)[i];
      a = (long long)__float_as_uint(fmaf(v.rh, v.rh, v.ih * v.ih));
    } else {
      a = nkey(cabs2(colp[i]));
    }
    if (better(a, i, best, bi)) { best = a; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const long long v2 = __shfl_xor_sync(0xffffffffu, best, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
    if (better(v2, i2, best, bi)) { best = v2; bi = i2; }
  }
  if (lane == 0) {
    const bool nonzero = DF ? (__uint_as_float((unsigned int)best) > 0.f) : (__longlong_as_double(best) > 0.0);
    const int p = nonzero ? bi : c;
    const int slot = c & 1;
    jb.la_p[slot] = p;
    jb.la_nz[slot] = nonzero ? 1 : 0;
    if constexpr (DF) {
      const dfc r = dfc_recip(reinterpret_cast<const dfc*>(colp)[p]);
      reinterpret_cast<dfc*>(jb.la_ip)[slot] = r;
    } else {
      const cplx d = colp[p];
      jb.la_ip[slot] = cabs2(d) > 0.0 ? cdiv(cmk(1.0, 0.0), d) : cmk(0.0, 0.0);
    }
  }
}

// Column c after step c (rows swapped): 1/d at row c, -u_i/d elsewhere.
__device__ __forceinline__ cplx final_pivot_col(const cplx* u, int i, int c, cplx ip) {
  if (i == c) return ip;
  const cplx v = u[i];
  return cmul(cmk(-v.x, -v.y), ip);
}

// smem: 2 x nmax pivot columns (ping-pong over the step parity), rows already swapped.
// DF: the eliminations run in double-float arithmetic on the FP32 pipes; the matrix is held
// in place as float pairs between a conversion pass at the start and one at the end, and
// pivots are chosen on |a|^2 to float precision.
template <bool DF>
__global__ void __launch_bounds__(kNT) k_pgj(const PgjJob* jobs, int nj, int nmax) {
  extern __shared__ cplx su[];
  __shared__ cplx s_ip[2];
  __shared__ dfc s_ipd[2];
  int jid = 0;
  while (jid + 1 < nj && jobs[jid + 1].b0 <= (int)blockIdx.x) ++jid;
  const PgjJob jb = jobs[jid];
  const int n = jb.n;
  const int lb = (int)blockIdx.x - jb.b0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gw = lb * kNW + warp, nw = jb.nb * kNW;
  cplx* A = jb.A;
  dfc* D = reinterpret_cast<dfc*>(jb.A);
  if constexpr (DF) {
    for (int j = gw; j < n; j += nw)
      for (int i = lane; i < n; i += 32) D[(int64_t)j * n + i] = to_dfc_bits(A[(int64_t)j * n + i]);
  }
  // the first pivot, by the owner of column 0 (the same warp converted that column)
  if (n > 0 && gw == 0) {
    __syncwarp();
    pgj_lookahead<DF>(jb, A, 0, lane);
  }
  if (group_sync(jb.gs, (unsigned)jb.nb) < 0) return;
  for (int c = 0; c < n; ++c) {
    {
      const int par = c & 1;
      // pivot row and 1/pivot found at the end of the previous step (lookahead)
      const int p = jb.la_p[par];
      const bool nonzero = jb.la_nz[par] != 0;
      if constexpr (DF) {
        dfc* u = reinterpret_cast<dfc*>(su) + (size_t)par * nmax;
        const dfc* colc = D + (int64_t)c * n;
        for (int i = tid; i < n; i += kNT) u[i] = colc[i];
        __syncthreads();
        if (tid == 0) {
          if (p != c) {
            const dfc t = u[c];
            u[c] = u[p];
            u[p] = t;
          }
          s_ipd[par] = reinterpret_cast<const dfc*>(jb.la_ip)[par];
        }
      } else {
        cplx* u = su + (size_t)par * nmax;
        const cplx* colc = A + (int64_t)c * n;
        for (int i = tid; i < n; i += kNT) u[i] = colc[i];
        __syncthreads();
        if (tid == 0) {
          if (p != c) {
            const cplx t = u[c];
            u[c] = u[p];
            u[p] = t;
          }
          s_ip[par] = jb.la_ip[par];
        }
      }
      if (tid == 0 && lb == 0) {
        jb.piv[c] = p;
        if (!nonzero) *jb.singular = 1;
      }
      __syncthreads();
      if constexpr (DF) {
        const dfc* u = reinterpret_cast<const dfc*>(su) + (size_t)par * nmax;
        const dfc* up = reinterpret_cast<const dfc*>(su) + (size_t)(1 - par) * nmax;
        const dfc ip = s_ipd[par];
        for (int j = gw; j < n; j += nw) {
          dfc* aj = D + (int64_t)j * n;
          if (j == c) continue;  // finalized at the next step (or after the last one)
          if (j == c - 1) {
            // deferred: the final values of column c-1 from step c-1 (1/d at row c-1, -u_i/d elsewhere)
            const dfc ipp = s_ipd[1 - par];
            for (int i = lane; i < n; i += 32) {
              if (i == c - 1) {
                aj[i] = ipp;
              } else {
                const dfc t = dfc_mul(up[i], ipp);
                aj[i] = {-t.rh, -t.rl, -t.ih, -t.il};
              }
            }
            __syncwarp();
          }
          const dfc ac = aj[p], ap = aj[c];  // rows c and p after the interchange
          const dfc r = dfc_mul(ac, ip);
          __syncwarp();
          for (int i = lane; i < n; i += 32) {
            if (i == c) continue;
            dfc x = (i == p) ? ap : aj[i];
            dfc_sub_mul(u[i], r, x);
            aj[i] = x;
          }
          if (lane == 0) aj[c] = r;
          if (j == c + 1) {  // the next pivot column is final for step c + 1
            __syncwarp();
            pgj_lookahead<true>(jb, reinterpret_cast<const cplx*>(aj), c + 1, lane);
          }
        }
      } else {
        const cplx* u = su + (size_t)par * nmax;
        const cplx* up = su + (size_t)(1 - par) * nmax;
        const cplx ip = s_ip[par];
        for (int j = gw; j < n; j += nw) {
          cplx* aj = A + (int64_t)j * n;
          if (j == c) continue;  // finalized at the next step (or after the last one)
          if (j == c - 1) {
            // deferred: the final values of column c-1 from step c-1
            const cplx ipp = s_ip[1 - par];
            for (int i = lane; i < n; i += 32) aj[i] = final_pivot_col(up, i, c - 1, ipp);
            __syncwarp();
          }
          const cplx ac = aj[p], ap = aj[c];  // rows c and p after the interchange
          const cplx r = cmul(ac, ip);
          __syncwarp();
          for (int i = lane; i < n; i += 32) {
            if (i == c) continue;
            const cplx x = (i == p) ? ap : aj[i];
            aj[i] = cfms(u[i], r, x);
          }
          if (lane == 0) aj[c] = r;
          if (j == c + 1) {  // the next pivot column is final for step c + 1
            __syncwarp();
            pgj_lookahead<false>(jb, aj, c + 1, lane);
          }
        }
      }
    }
    if (group_sync(jb.gs, (unsigned)jb.nb) < 0) return;
  }
  // the last pivot column of this matrix
  if (n > 0) {
    const int c = n - 1;
    const int own = c % nw;
    if (own == gw) {
      if constexpr (DF) {
        const dfc* u = reinterpret_cast<const dfc*>(su) + (size_t)(c & 1) * nmax;
        const dfc ip = s_ipd[c & 1];
        dfc* ac = D + (int64_t)c * n;
        for (int i = lane; i < n; i += 32) {
          if (i == c) {
            ac[i] = ip;
          } else {
            const dfc t = dfc_mul(u[i], ip);
            ac[i] = {-t.rh, -t.rl, -t.ih, -t.il};
          }
        }
      } else {
        const cplx* u = su + (size_t)(c & 1) * nmax;
        const cplx ip = s_ip[c & 1];
        cplx* ac = A + (int64_t)c * n;
        for (int i = lane; i < n; i += 32) ac[i] = final_pivot_col(u, i, c, ip);
      }
    }
  }
  if constexpr (DF) {
    __syncwarp();
    // every column's final values were written by its owning warp: convert them back
    for (int j = gw; j < n; j += nw)
      for (int i = lane; i < n; i += 32) A[(int64_t)j * n + i] = from_dfc_bits(D[(int64_t)j * n + i]);
  }
}

// tmp(:, j) = A(:, src[j]) where src undoes the row interchanges (column swaps
// (c, piv[c]) in reverse order); then A = tmp (k_pgj_copy).
__global__ void __launch_bounds__(kNT) k_pgj_unpivot(const PgjJob* jobs, int nmax) {
  extern __shared__ int src[];
  const PgjJob jb = jobs[blockIdx.y];
  const int n = jb.n;
  if (threadIdx.x == 0) {
    for (int q = 0; q < n; ++q) src[q] = q;
    for (int c = n - 1; c >= 0; --c) {
      const int p = jb.piv[c];
      const int t = src[c];
      src[c] = src[p];
      src[p] = t;
    }
  }
  __syncthreads();
  const int64_t tot = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)kNT + threadIdx.x; e < tot; e += (int64_t)gridDim.x * kNT) {
    const int i = (int)(e % n), j = (int)(e / n);
    jb.tmp[e] = jb.A[(int64_t)src[j] * n + i];
  }
}

__global__ void k_pgj_copy(const PgjJob* jobs) {
  const PgjJob jb = jobs[blockIdx.y];
  const int64_t tot = (int64_t)jb.n * jb.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
    jb.A[e] = jb.tmp[e];
}

}  // namespace

template <bool DF>
static int pgj_grid(size_t smem) {
  static const int sms = [] {
    int dev = 0, sm = 0;
    HBS_CUDA(cudaGetDevice(&dev));
    HBS_CUDA(cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev));
    return sm;
  }();
  HBS_CUDA(raise_smem_limit((const void*)k_pgj<DF>, smem));
  int per_sm = 0;
  HBS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pgj<DF>, kNT, smem));
  if (per_sm < 1) throw Error(HBS_ERR_CUDA, "persistent Gauss-Jordan kernel does not fit on an SM");
  return sms * std::min(per_sm, 2);
}

// In-place inverses of the matrices (pointer, n) in one persistent launch; throws
// HBS_WARN_ILLCOND on a singular block.
void pgj_run(const std::vector<std::pair<cplx*, int>>& mats, cudaStream_t s, const char* what) {
  const int nj = (int)mats.size();
  if (nj == 0) return;
  int nmax = 0;
  double work = 0.0, fl = 0.0;
  int64_t ptot = 0, atot = 0;
  for (const auto& m : mats) {
    nmax = std::max(nmax, m.second);
    work += (double)m.second * m.second;
    fl += 8.0 * (double)m.second * m.second * m.second;
    ptot += m.second;
    atot += (int64_t)m.second * m.second;
  }
  const size_t smem = 2 * (size_t)nmax * sizeof(cplx);
  // double-float eliminations on handles built with double-float precision
  const bool df = gemm_double_float();
  const int G = df ? pgj_grid<true>(smem) : pgj_grid<false>(smem);
  if (nj > G) throw Error(HBS_ERR_INTERNAL, "persistent Gauss-Jordan batch larger than the grid");
  // CTAs per matrix in proportion to its size, at least one each.
  std::vector<int> nb(nj, 1);
  const int left = G - nj;
  for (int j = 0; j < nj; ++j)
    nb[j] += (int)std::floor((double)left * mats[j].second * mats[j].second / work);
  int used = 0;
  for (int v : nb) used += v;
  for (int j = 0; used < G; j = (j + 1) % nj, ++used) ++nb[j];
  DevBuf<int> piv(ptot), sing(nj), la_p(2 * nj), la_nz(2 * nj);
  DevBuf<cplx> la_ip(2 * nj);
  DevBuf<cplx> tmp(atot);
  DevBuf<GridSync> gs(nj);
  HBS_CUDA(cudaMemsetAsync(sing.get(), 0, sizeof(int) * nj, s));
  HBS_CUDA(cudaMemsetAsync(gs.get(), 0, sizeof(GridSync) * nj, s));
  std::vector<PgjJob> jobs(nj);
  int64_t po = 0, ao = 0;
  int b0 = 0;
  for (int j = 0; j < nj; ++j) {
    jobs[j] = {mats[j].first, mats[j].second, b0,  nb[j], piv.get() + po, sing.get() + j, tmp.get() + ao,
               la_p.get() + 2 * j, la_nz.get() + 2 * j, la_ip.get() + 2 * j, gs.get() + j};
    po += mats[j].second;
    ao += (int64_t)mats[j].second * mats[j].second;
    b0 += nb[j];
  }
  DevBuf<PgjJob> dj;
  dj.upload(jobs, s);
  std::vector<int> hs(nj);
  std::vector<GridSync> hg(nj);
  {
    const PgjJob* a0 = dj.get();
    int a1 = nj, a2 = nmax;
    void* args[] = {&a0, &a1, &a2};
    std::lock_guard<std::mutex> lock(coop_mutex());
    {
      prof::KScope _ks("k_pgj", s, fl, 0.0);
      const void* fn = df ? (const void*)k_pgj<true> : (const void*)k_pgj<false>;
      HBS_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kNT), args, smem, s));
    }
    HBS_LAUNCH_CHECK("k_pgj");
    read_to_host(hg.data(), gs.get(), sizeof(GridSync) * nj, s);
  }
  for (const auto& g : hg)
    if (g.timed_out) throw Error(HBS_ERR_TIMEOUT, "persistent Gauss-Jordan: a barrier wait gave up");
  {
    prof::KScope _ks("k_pgj_unpivot", s);
    const size_t sm = (size_t)nmax * sizeof(int);
    HBS_CUDA(raise_smem_limit((const void*)k_pgj_unpivot, sm));
    k_pgj_unpivot<<<dim3(std::max(1, 1216 / nj), nj), kNT, sm, s>>>(dj.get(), nmax);
    k_pgj_copy<<<dim3(std::max(1, 1216 / nj), nj), 256, 0, s>>>(dj.get());
  }
  HBS_LAUNCH_CHECK("k_pgj_unpivot");
  read_to_host(hs.data(), sing.get(), sizeof(int) * nj, s);
  for (int j = 0; j < nj; ++j)
    if (hs[j]) throw Error(HBS_WARN_ILLCOND, std::string("singular block in ") + what);
}

}  // namespace hbs
