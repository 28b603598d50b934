// Batched variable-size complex FP64 GEMM: C = alpha * op(A) * B + beta * C for a
// list of jobs of different shapes (one grid, jobs x tiles).  Used for the level-wise
// products of the HBS inversion (Eqs. woodbury, def_muhD..def_muG) and the telescoping
// apply of the compressed inverse (Sec. 4).
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

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
  int transC;            // 1: C stored row-major, C(i, j) at C[i ldc + j]
  int a_real_digits = 0; // tensor-core products: 0 for a general A; d > 0 when A is real and each
                         // of its rows needs only its first d digit planes (e.g. 1 for signs)
};

constexpr int GBM = 32, GBN = 32, GBK = 8;

// The multiply-adds of one GBK slice for one thread's outputs (rows tr, tr + 16; columns tc,
// tc + 16), leaving out the second row (R1 false) or column (C1 false).
template <bool R1, bool C1>
__device__ __forceinline__ void tile_fma(const cplx (*As)[GBM + 1], const cplx (*Bs)[GBN + 1], int tr, int tc,
                                         cplx (&acc)[2][2]) {
#pragma unroll
  for (int kk = 0; kk < GBK; ++kk) {
    const cplx a0 = As[kk][tr], b0 = Bs[kk][tc];
    acc[0][0] = cfma(a0, b0, acc[0][0]);
    if (C1) {
      const cplx b1 = Bs[kk][tc + 16];
      acc[0][1] = cfma(a0, b1, acc[0][1]);
      if (R1) acc[1][1] = cfma(As[kk][tr + 16], b1, acc[1][1]);
    }
    if (R1) acc[1][0] = cfma(As[kk][tr + 16], b0, acc[1][0]);
  }
}

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
  // Output columns tc and tc + 16, rows tr and tr + 16 of the tile: a warp holds two values
  // of tc and all 16 of tr, so for narrow products whole warps skip the multiply-adds of
  // columns past n, and every warp those of rows past m when the tile has at most 16 (a warp
  // instruction costs the same however many of its lanes are active).
  const bool c0 = col0 + tc < n, c1 = col0 + tc + 16 < n, r1 = row0 + 16 < m;
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
    if (c0) {
      if (c1) {
        if (r1) tile_fma<true, true>(As, Bs, tr, tc, acc);
        else tile_fma<false, true>(As, Bs, tr, tc, acc);
      } else {
        if (r1) tile_fma<true, false>(As, Bs, tr, tc, acc);
        else tile_fma<false, false>(As, Bs, tr, tc, acc);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int gr = row0 + tr + 16 * a, gc = col0 + tc + 16 * b;
      if (gr < m && gc < n) {
        cplx* c = jb.transC ? jb.C + (int64_t)gr * jb.ldc + gc : jb.C + (int64_t)gc * jb.ldc + gr;
        cplx v = cmul(jb.alpha, acc[a][b]);
        if (jb.beta.x != 0.0 || jb.beta.y != 0.0) v = cfma(jb.beta, *c, v);
        *c = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Double-float variant.  FP64 operands are split on load into float pairs (hi, lo),
// hi = fl32(x), lo = fl32(x - hi), and every multiply-add is carried out in double-float
// arithmetic on the FP32 pipes (error-free product via fmaf, error-free sum via two-sum,
// about 48 significant bits).  GB300 issues FP32 FMAs at 64x its FP64 rate, so the
// double-float product is several times faster than DFMA while keeping relative
// errors near 2^-48 per operation; results are written back in FP64.
// ---------------------------------------------------------------------------
// acc += a b in double-float (re += ar br - ai bi; im += ar bi + ai br), lazy low parts.
__device__ __forceinline__ void dfc_mac_tile(const dfc& a, const dfc& b, dfc& c) {
  df_mac(a.rh, a.rl, b.rh, b.rl, c.rh, c.rl);
  df_mac(-a.ih, -a.il, b.ih, b.il, c.rh, c.rl);
  df_mac(a.rh, a.rl, b.ih, b.il, c.ih, c.il);
  df_mac(a.ih, a.il, b.rh, b.rl, c.ih, c.il);
}

// The double-float multiply-adds of one GBK slice for one thread's outputs, leaving out the
// second row (R1 false) or column (C1 false).
// The slice loop is unrolled by 2: fully unrolled (8), the four variants' code (48 FP32-pipe
// instructions per complex multiply-add) overflows the instruction cache and the warps stall on
// instruction fetches; not unrolled at all, the loop overhead shows.
template <bool R1, bool C1>
__device__ __forceinline__ void tile_mac_df(const dfc (*As)[GBM + 1], const dfc (*Bs)[GBN + 1], int tr, int tc,
                                            dfc (&acc)[2][2]) {
#pragma unroll 2
  for (int kk = 0; kk < GBK; ++kk) {
    const dfc a0 = As[kk][tr], b0 = Bs[kk][tc];
    dfc_mac_tile(a0, b0, acc[0][0]);
    if (C1) {
      const dfc b1 = Bs[kk][tc + 16];
      dfc_mac_tile(a0, b1, acc[0][1]);
      if (R1) dfc_mac_tile(As[kk][tr + 16], b1, acc[1][1]);
    }
    if (R1) dfc_mac_tile(As[kk][tr + 16], b0, acc[1][0]);
  }
}

// Slices are double-buffered in shared memory: while the CTA multiplies one slice, each thread
// already holds its elements of the next in registers (loads issued before the multiply-adds),
// and stores them into the other buffer afterwards, so one barrier per slice suffices and the
// L2 latency of the loads overlaps the arithmetic.
static __global__ void __launch_bounds__(256) k_zgemm_batched_df(const GemmJob* jobs, int njobs) {
  __shared__ dfc As[2][GBK][GBM + 1];
  __shared__ dfc Bs[2][GBK][GBN + 1];
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
  const int tr = tid & 15, tc = tid >> 4;
  dfc acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = {0.f, 0.f, 0.f, 0.f};
  const int m = jb.m, n = jb.n, K = jb.k;
  // the same skipping of padded rows and columns as in k_zgemm_batched
  const bool c0 = col0 + tc < n, c1 = col0 + tc + 16 < n, r1 = row0 + 16 < m;
  // this thread's element of each slice: A (row ar, slice column ak), B (slice row bk, column bc)
  const bool ta = jb.transA != 0;
  const int ar = ta ? tid >> 3 : tid & 31, ak = ta ? tid & 7 : tid >> 5;
  const int bc = tid >> 3, bk = tid & 7;
  const bool a_row = row0 + ar < m, b_col = col0 + bc < n;
  const cplx* pa = ta ? jb.A + (int64_t)(row0 + ar) * jb.lda + ak : jb.A + (int64_t)ak * jb.lda + row0 + ar;
  const int64_t a_step = ta ? GBK : (int64_t)GBK * jb.lda;
  const cplx* pb = jb.B + (int64_t)(col0 + bc) * jb.ldb + bk;
  cplx av = (a_row && ak < K) ? pa[0] : cmk(0.0, 0.0);
  cplx bv = (b_col && bk < K) ? pb[0] : cmk(0.0, 0.0);
  As[0][ak][ar] = to_dfc_bits(av);
  Bs[0][bk][bc] = to_dfc_bits(bv);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += GBK) {
    const int k1 = k0 + GBK;
    const bool more = k1 < K;
    if (more) {
      pa += a_step;
      pb += GBK;
      av = (a_row && k1 + ak < K) ? pa[0] : cmk(0.0, 0.0);
      bv = (b_col && k1 + bk < K) ? pb[0] : cmk(0.0, 0.0);
    }
    if (c0) {
      if (c1) {
        if (r1) tile_mac_df<true, true>(As[buf], Bs[buf], tr, tc, acc);
        else tile_mac_df<false, true>(As[buf], Bs[buf], tr, tc, acc);
      } else {
        if (r1) tile_mac_df<true, false>(As[buf], Bs[buf], tr, tc, acc);
        else tile_mac_df<false, false>(As[buf], Bs[buf], tr, tc, acc);
      }
    }
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        df_norm(acc[x][y].rh, acc[x][y].rl);
        df_norm(acc[x][y].ih, acc[x][y].il);
      }
    if (more) {
      As[buf ^ 1][ak][ar] = to_dfc_bits(av);
      Bs[buf ^ 1][bk][bc] = to_dfc_bits(bv);
    }
    __syncthreads();
    buf ^= 1;
  }
  const bool unit_alpha = jb.alpha.x == 1.0 && jb.alpha.y == 0.0;
  const bool minus_alpha = jb.alpha.x == -1.0 && jb.alpha.y == 0.0;
  const bool zero_beta = jb.beta.x == 0.0 && jb.beta.y == 0.0;
  const bool unit_beta = jb.beta.x == 1.0 && jb.beta.y == 0.0;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int gr = row0 + tr + 16 * a, gc = col0 + tc + 16 * b;
      if (gr < m && gc < n) {
        cplx* c = jb.transC ? jb.C + (int64_t)gr * jb.ldc + gc : jb.C + (int64_t)gc * jb.ldc + gr;
        const dfc& q = acc[a][b];
        // the common (alpha, beta) = (1, 0) and (-1, 1) take two or four FP64 adds only
        const cplx sum = cmk(f2d_bits(q.rh) + f2d_bits(q.rl), f2d_bits(q.ih) + f2d_bits(q.il));
        cplx v;
        if (unit_alpha && zero_beta) {
          v = sum;
        } else if (minus_alpha && unit_beta) {
          v = csub(*c, sum);
        } else {
          v = cmul(jb.alpha, sum);
          if (!zero_beta) v = cfma(jb.beta, *c, v);
        }
        *c = v;
      }
    }
  }
}

// Host helper: fill tile bookkeeping and return the total tile count.
inline int64_t gemm_plan(GemmJob* jobs, int njobs, int bm = GBM, int bn = GBN) {
  int64_t tot = 0;
  for (int i = 0; i < njobs; ++i) {
    jobs[i].tiles_m = (jobs[i].m + bm - 1) / bm;
    jobs[i].tiles_n = (jobs[i].n + bn - 1) / bn;
    if (jobs[i].m <= 0 || jobs[i].n <= 0) { jobs[i].tiles_m = 0; jobs[i].tiles_n = 0; }
    jobs[i].tile_base = (int)tot;
    tot += (int64_t)jobs[i].tiles_m * jobs[i].tiles_n;
  }
  return tot;
}

}  // namespace hbs
