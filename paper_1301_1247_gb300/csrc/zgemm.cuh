// Batched variable-size complex FP64 GEMM: C = alpha * op(A) * B + beta * C for a
// list of jobs of different shapes (one grid, jobs x tiles).  Used for the level-wise
// products of the HBS inversion (Eqs. woodbury, def_muhD..def_muG) and the telescoping
// apply of the compressed inverse (Sec. 4).
#pragma once

#include "common.cuh"

namespace hbs {

struct GemmJob {
  const cplx* A;
  const cplx* B;
  cplx* C;
  int m, n, k;
  int lda, ldb, ldc;
  cplx alpha, beta;
  int tiles_m, tiles_n;  // ceil(m / BM), ceil(n / BN)
  int tile_base;         // prefix sum of tiles over earlier jobs
  int transA;            // 1: op(A) = A^T (A stored k x m, column-major, leading dimension lda)
};

constexpr int GBM = 32, GBN = 32, GBK = 8;

// grid.x = total tiles over all jobs; each CTA finds its job by binary search on tile_base.
static __global__ void __launch_bounds__(256) k_zgemm_batched(const GemmJob* jobs, int njobs) {
  __shared__ cplx As[GBK][GBM + 1];
  __shared__ cplx Bs[GBK][GBN + 1];
  int t = blockIdx.x;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  const GemmJob& jb = jobs[lo];
  t -= jb.tile_base;
  const int tm = t % jb.tiles_m, tn = t / jb.tiles_m;
  const int row0 = tm * GBM, col0 = tn * GBN;
  const int tid = threadIdx.x;
  const int tr = tid & 15, tc = tid >> 4;  // 16 x 16 threads, 2 x 2 outputs each
  cplx acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = cmk(0.0, 0.0);
  const int m = jb.m, n = jb.n, K = jb.k;
  for (int k0 = 0; k0 < K; k0 += GBK) {
    // load A tile (GBM x GBK): 256 threads, one element each
    {
      if (jb.transA) {
        int r = tid >> 3, kk = tid & 7;
        int gr = row0 + r, gk = k0 + kk;
        As[kk][r] = (gr < m && gk < K) ? jb.A[(int64_t)gr * jb.lda + gk] : cmk(0.0, 0.0);
      } else {
        int r = tid & 31, kk = tid >> 5;
        int gr = row0 + r, gk = k0 + kk;
        As[kk][r] = (gr < m && gk < K) ? jb.A[(int64_t)gk * jb.lda + gr] : cmk(0.0, 0.0);
      }
      int c = tid >> 3, kb = tid & 7;
      int gc = col0 + c, gkb = k0 + kb;
      Bs[kb][c] = (gc < n && gkb < K) ? jb.B[(int64_t)gc * jb.ldb + gkb] : cmk(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      cplx a0 = As[kk][tr], a1 = As[kk][tr + 16];
      cplx b0 = Bs[kk][tc], b1 = Bs[kk][tc + 16];
      acc[0][0] = cfma(a0, b0, acc[0][0]);
      acc[0][1] = cfma(a0, b1, acc[0][1]);
      acc[1][0] = cfma(a1, b0, acc[1][0]);
      acc[1][1] = cfma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int gr = row0 + tr + 16 * a, gc = col0 + tc + 16 * b;
      if (gr < m && gc < n) {
        cplx* c = jb.C + (int64_t)gc * jb.ldc + gr;
        cplx v = cmul(jb.alpha, acc[a][b]);
        if (jb.beta.x != 0.0 || jb.beta.y != 0.0) v = cfma(jb.beta, *c, v);
        *c = v;
      }
    }
  }
}

// Host helper: fill tile bookkeeping and return the total tile count.
inline int64_t gemm_plan(GemmJob* jobs, int njobs) {
  int64_t tot = 0;
  for (int i = 0; i < njobs; ++i) {
    jobs[i].tiles_m = (jobs[i].m + GBM - 1) / GBM;
    jobs[i].tiles_n = (jobs[i].n + GBN - 1) / GBN;
    if (jobs[i].m <= 0 || jobs[i].n <= 0) { jobs[i].tiles_m = 0; jobs[i].tiles_n = 0; }
    jobs[i].tile_base = (int)tot;
    tot += (int64_t)jobs[i].tiles_m * jobs[i].tiles_n;
  }
  return tot;
}

}  // namespace hbs
