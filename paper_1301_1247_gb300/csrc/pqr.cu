// Persistent column-pivoted Householder QR for interpolative decompositions (Def. 3.1)
// of large matrices: one cooperative launch runs every pivot step of every matrix in a
// batch, with one grid barrier per step, instead of three launches per step.
//
// Step s of a matrix (m x n, column-major, columns = the members to choose from):
//   * every CTA of the matrix reduces the per-CTA partial maxima of the column norms
//     left by step s-1 and finds the pivot column p (largest remaining norm, lowest index
//     on ties) - the same reduction in every CTA, so all agree bit for bit;
//   * every CTA forms the reflector of column p (rows s..m-1) in shared memory;
//   * each active column j != p is owned by one warp and is updated (in registers for
//     its first 64 rows, the rest streamed 4 rows per lane at a time), its norm downdated (recomputed on cancellation), and the
//     CTA's partial maximum for step s+1 recorded.
// Columns are never swapped: pivot p of step s stays where it is, its rows < s hold
// R(:, s) and its rows > s the reflector tail; the diagonal beta_s, the reflector head
// v0_s and tau_s go to per-step arrays.  The row ID's permutation is the one the
// column-swapping algorithm would produce, and T = R11^{-1} R12 follows from one
// triangular solve per column.
#include <algorithm>
#include <cstdio>

#include "balance.hpp"
#include "dense_kernels.cuh"
#include "dfloat.cuh"
#include "gridsync.cuh"
#include "profile.hpp"
#include "qp_kernels.cuh"

namespace hbs {

namespace {

constexpr int kNT = 256;
constexpr int kNW = kNT / 32;
constexpr int kReg = 2;   // rows per lane held in registers between the two passes of an update
constexpr int kU = 4;     // rows per lane loaded together in the streamed part (loads in flight)

// L1 prefetch of the lane's next kU rows (in-bounds rows only): another chunk in flight
// without holding registers for it.
template <typename T>
__device__ __forceinline__ void prefetch_next(const T* aj, int64_t i0, int64_t stride, int64_t m) {
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int64_t ip = i0 + stride * (kU + u);
    if (ip < m) asm volatile("prefetch.L1 [%0];" ::"l"(aj + ip));
  }
}

struct PqrJob {
  cplx* A;
  int64_t m, n;
  int kcap;
  int b0, nb;  // CTA range of this matrix
  int gw;      // warps per column (1, 2, 4, 8)
  double* nrm;
  double* nref;
  int* piv;
  cplx* beta;
  cplx* v0;
  double* tau;
  PqrState* st;
  int* perm;
  cplx* T;
  cplx* r11r;  // k x k row-major copy of R11 (scratch for the triangular solves)
  cplx* r11c;  // k x k column-major copy of R11
  cplx* invd;  // 1 / R_ii (k)
  int* pos;    // n: position of each column in perm (scratch)
  GridSync* gs;  // barrier of this matrix's CTAs
};

template <int NT>
__device__ __forceinline__ cplx block_sum_c(cplx v, double* red) {
  double a = block_sum<NT>(v.x, red);
  double b = block_sum<NT>(v.y, red);
  return cmk(a, b);
}

// Warp sum of a complex value with five FP64 additions instead of ten: after the first
// exchange the lower half-warp carries real parts and the upper half imaginary parts.
// The pairs added are those of the plain butterfly, so the sum is bitwise the same.
__device__ __forceinline__ cplx warp_sum_c(cplx w) {
  const bool lo = (threadIdx.x & 31) < 16;
  double keep = lo ? w.x : w.y;
  keep += __shfl_xor_sync(0xffffffffu, lo ? w.y : w.x, 16);
  for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
  return cmk(__shfl_sync(0xffffffffu, keep, 0), __shfl_sync(0xffffffffu, keep, 16));
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// x = R^{-1} b for upper-triangular R (k x k, row-major), one warp; x is written to
// global memory row by row (x may alias b: b[i] is read before x[i] is written).
__device__ __forceinline__ void tsolve_row_major(const cplx* R, int k, const cplx* b, cplx* x, int lane) {
  for (int i = k - 1; i >= 0; --i) {
    const cplx* ri = R + (int64_t)i * k;
    cplx acc = cmk(0.0, 0.0);
    for (int l = i + 1 + lane; l < k; l += 32) acc = cfma(ri[l], x[l], acc);
    acc = warp_sum_c(acc);
    if (lane == 0) x[i] = cdiv(csub(b[i], acc), ri[i]);
    __syncwarp();
  }
}

// One Householder update of column j at step s: the 32 lanes of a warp own the column,
// its first 32 kReg rows below s stay in registers between the two passes and the rest
// (tall matrices) is streamed twice, kU rows per lane loaded together so that the loads
// overlap instead of each waiting on the accumulation chain.  Each lane still adds its rows
// in increasing order, so the sums do not depend on kU.
__device__ __forceinline__ double update_col_warp(cplx* aj, const cplx* vt, int64_t m, int64_t s, cplx v0, double tau,
                                                  double nj, double* nref_j, int lane) {
  cplx r[kReg];
  cplx w = cmk(0.0, 0.0);
#pragma unroll
  for (int q = 0; q < kReg; ++q) {
    const int64_t i = s + 1 + lane + 32 * q;
    if (i < m) {
      r[q] = aj[i];
      w = cfma(cconj(vt[i - s - 1]), r[q], w);
    }
  }
  for (int64_t i0 = s + 1 + lane + 32 * kReg; i0 < m; i0 += 32 * kU) {
    prefetch_next(aj, i0, 32, m);
    cplx a[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + 32 * u < m) a[u] = aj[i0 + 32 * u];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + 32 * u < m) w = cfma(cconj(vt[i0 + 32 * u - s - 1]), a[u], w);
  }
  w = warp_sum_c(w);
  const cplx ajs = aj[s];
  w = cscale(cfma(cconj(v0), ajs, w), tau);
  const cplx top = cfms(v0, w, ajs);
#pragma unroll
  for (int q = 0; q < kReg; ++q) {
    const int64_t i = s + 1 + lane + 32 * q;
    if (i < m) {
      r[q] = cfms(vt[i - s - 1], w, r[q]);
      aj[i] = r[q];
    }
  }
  for (int64_t i0 = s + 1 + lane + 32 * kReg; i0 < m; i0 += 32 * kU) {
    prefetch_next(aj, i0, 32, m);
    cplx a[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + 32 * u < m) a[u] = aj[i0 + 32 * u];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + 32 * u < m) aj[i0 + 32 * u] = cfms(vt[i0 + 32 * u - s - 1], w, a[u]);
  }
  double t = nj - cabs2(top);
  if (t <= 0.0078125 * *nref_j) {
    // cancellation: recompute the norm of rows s+1.. from the updated values
    double q2 = 0.0;
#pragma unroll
    for (int q = 0; q < kReg; ++q)
      if (s + 1 + lane + 32 * q < m) q2 += cabs2(r[q]);
    for (int64_t i = s + 1 + lane + 32 * kReg; i < m; i += 32) q2 += cabs2(aj[i]);
    t = warp_sum(q2);
    if (lane == 0) *nref_j = t;
  }
  __syncwarp();
  if (lane == 0) aj[s] = top;
  return t;
}

__device__ __forceinline__ void group_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// The same update by a group of GW warps (rows split over the group's 32 GW lanes): for the
// top tree levels, whose few columns would otherwise leave most warps idle.  The group's
// partial sums meet in shared memory (slot alternates per column) behind a named barrier.
__device__ double update_col_group(cplx* aj, const cplx* vt, int64_t m, int64_t s, cplx v0, double tau, double nj,
                                   double* nref_j, int gl, int GW, int grp, int wg, int lane, int slot, cplx* redc,
                                   double* redn) {
  const int64_t stride = 32 * GW;
  const int base = slot * kNW + grp * GW;
  const cplx ajs = aj[s];  // read by every warp before the group's first barrier
  cplx r[kReg];
  cplx w = cmk(0.0, 0.0);
#pragma unroll
  for (int q = 0; q < kReg; ++q) {
    const int64_t i = s + 1 + gl + stride * q;
    if (i < m) {
      r[q] = aj[i];
      w = cfma(cconj(vt[i - s - 1]), r[q], w);
    }
  }
  for (int64_t i0 = s + 1 + gl + stride * kReg; i0 < m; i0 += stride * kU) {
    prefetch_next(aj, i0, stride, m);
    cplx a[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + stride * u < m) a[u] = aj[i0 + stride * u];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + stride * u < m) w = cfma(cconj(vt[i0 + stride * u - s - 1]), a[u], w);
  }
  w = warp_sum_c(w);
  if (lane == 0) redc[base + wg] = w;
  group_barrier(1 + grp, 32 * GW);
  cplx tot = cmk(0.0, 0.0);
  for (int k = 0; k < GW; ++k) tot = cadd(tot, redc[base + k]);
  w = cscale(cfma(cconj(v0), ajs, tot), tau);
  const cplx top = cfms(v0, w, ajs);
#pragma unroll
  for (int q = 0; q < kReg; ++q) {
    const int64_t i = s + 1 + gl + stride * q;
    if (i < m) {
      r[q] = cfms(vt[i - s - 1], w, r[q]);
      aj[i] = r[q];
    }
  }
  for (int64_t i0 = s + 1 + gl + stride * kReg; i0 < m; i0 += stride * kU) {
    prefetch_next(aj, i0, stride, m);
    cplx a[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + stride * u < m) a[u] = aj[i0 + stride * u];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + stride * u < m) aj[i0 + stride * u] = cfms(vt[i0 + stride * u - s - 1], w, a[u]);
  }
  double t = nj - cabs2(top);
  if (t <= 0.0078125 * *nref_j) {  // uniform over the group
    double q2 = 0.0;
#pragma unroll
    for (int q = 0; q < kReg; ++q)
      if (s + 1 + gl + stride * q < m) q2 += cabs2(r[q]);
    for (int64_t i = s + 1 + gl + stride * kReg; i < m; i += stride) q2 += cabs2(aj[i]);
    q2 = warp_sum(q2);
    if (lane == 0) redn[base + wg] = q2;
    group_barrier(1 + grp, 32 * GW);
    t = 0.0;
    for (int k = 0; k < GW; ++k) t += redn[base + k];
    if (gl == 0) *nref_j = t;
  }
  if (gl == 0) aj[s] = top;
  return t;
}

// ---- double-float updates (handles built with double-float precision) ----
// From the norm pass to the end of the launch the matrix is held in place as complex
// double-float (dfc, 16 bytes like the complex double it replaces), and the rank-one
// updates, which carry almost all of the work, run on the FP32 pipes.  Column norms,
// pivot choices and the reflector scalars stay FP64.

// w = tau (conj(v0) a_s + tot) and the new row-s entry top = a_s - v0 w.
__device__ __forceinline__ void df_col_scalars(const dfc& ajs, const dfc& tot, const dfc& v0, float th, float tl,
                                               dfc* w, dfc* top) {
  dfc u = tot;
  dfc_cdot_acc(v0, ajs, u);
  dfc_norm(u);
  *w = dfc_scale(th, tl, u);
  dfc t = ajs;
  dfc_sub_mul(v0, *w, t);
  *top = t;
}

// Downdated squared norm nj - |top|^2 (FP64).
__device__ __forceinline__ double df_downdate(double nj, const dfc& top) {
  float qh = 0.f, ql = 0.f;
  df_abs2_acc(top, qh, ql);
  return (nj - f2d_bits(qh)) - f2d_bits(ql);
}

__device__ __forceinline__ double update_col_warp_df(dfc* aj, const dfc* vt, int64_t m, int64_t s, const dfc& v0,
                                                     float th, float tl, double nj, double* nref_j, int lane) {
  dfc r[kReg];
  dfc w = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < kReg; ++q) {
    const int64_t i = s + 1 + lane + 32 * q;
    if (i < m) {
      r[q] = aj[i];
      dfc_cdot_acc(vt[i - s - 1], r[q], w);
    }
  }
  for (int64_t i0 = s + 1 + lane + 32 * kReg; i0 < m; i0 += 32 * kU) {
    prefetch_next(aj, i0, 32, m);
    dfc a[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + 32 * u < m) a[u] = aj[i0 + 32 * u];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + 32 * u < m) dfc_cdot_acc(vt[i0 + 32 * u - s - 1], a[u], w);
  }
  w = dfc_warp_sum(w);
  const dfc ajs = aj[s];
  dfc wv, top;
  df_col_scalars(ajs, w, v0, th, tl, &wv, &top);
#pragma unroll
  for (int q = 0; q < kReg; ++q) {
    const int64_t i = s + 1 + lane + 32 * q;
    if (i < m) {
      dfc_sub_mul(vt[i - s - 1], wv, r[q]);
      aj[i] = r[q];
    }
  }
  for (int64_t i0 = s + 1 + lane + 32 * kReg; i0 < m; i0 += 32 * kU) {
    prefetch_next(aj, i0, 32, m);
    dfc a[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + 32 * u < m) a[u] = aj[i0 + 32 * u];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + 32 * u < m) {
        dfc_sub_mul(vt[i0 + 32 * u - s - 1], wv, a[u]);
        aj[i0 + 32 * u] = a[u];
      }
  }
  double t = df_downdate(nj, top);
  if (t <= 0.0078125 * *nref_j) {
    float qh = 0.f, ql = 0.f;
#pragma unroll
    for (int q = 0; q < kReg; ++q)
      if (s + 1 + lane + 32 * q < m) df_abs2_acc(r[q], qh, ql);
    for (int64_t i = s + 1 + lane + 32 * kReg; i < m; i += 32) df_abs2_acc(aj[i], qh, ql);
    t = warp_sum(f2d_bits(qh) + f2d_bits(ql));
    if (lane == 0) *nref_j = t;
  }
  __syncwarp();
  if (lane == 0) aj[s] = top;
  return t;
}

__device__ double update_col_group_df(dfc* aj, const dfc* vt, int64_t m, int64_t s, const dfc& v0, float th, float tl,
                                      double nj, double* nref_j, int gl, int GW, int grp, int wg, int lane, int slot,
                                      dfc* redc, double* redn) {
  const int64_t stride = 32 * GW;
  const int base = slot * kNW + grp * GW;
  const dfc ajs = aj[s];  // read by every warp before the group's first barrier
  dfc r[kReg];
  dfc w = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < kReg; ++q) {
    const int64_t i = s + 1 + gl + stride * q;
    if (i < m) {
      r[q] = aj[i];
      dfc_cdot_acc(vt[i - s - 1], r[q], w);
    }
  }
  for (int64_t i0 = s + 1 + gl + stride * kReg; i0 < m; i0 += stride * kU) {
    prefetch_next(aj, i0, stride, m);
    dfc a[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + stride * u < m) a[u] = aj[i0 + stride * u];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + stride * u < m) dfc_cdot_acc(vt[i0 + stride * u - s - 1], a[u], w);
  }
  w = dfc_warp_sum(w);
  if (lane == 0) redc[base + wg] = w;
  group_barrier(1 + grp, 32 * GW);
  dfc tot = {0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < GW; ++k) {
    const dfc p = redc[base + k];
    df_add_to(p.rh, p.rl, tot.rh, tot.rl);
    df_add_to(p.ih, p.il, tot.ih, tot.il);
  }
  dfc_norm(tot);
  dfc wv, top;
  df_col_scalars(ajs, tot, v0, th, tl, &wv, &top);
#pragma unroll
  for (int q = 0; q < kReg; ++q) {
    const int64_t i = s + 1 + gl + stride * q;
    if (i < m) {
      dfc_sub_mul(vt[i - s - 1], wv, r[q]);
      aj[i] = r[q];
    }
  }
  for (int64_t i0 = s + 1 + gl + stride * kReg; i0 < m; i0 += stride * kU) {
    prefetch_next(aj, i0, stride, m);
    dfc a[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + stride * u < m) a[u] = aj[i0 + stride * u];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + stride * u < m) {
        dfc_sub_mul(vt[i0 + stride * u - s - 1], wv, a[u]);
        aj[i0 + stride * u] = a[u];
      }
  }
  double t = df_downdate(nj, top);
  if (t <= 0.0078125 * *nref_j) {  // uniform over the group
    float qh = 0.f, ql = 0.f;
#pragma unroll
    for (int q = 0; q < kReg; ++q)
      if (s + 1 + gl + stride * q < m) df_abs2_acc(r[q], qh, ql);
    for (int64_t i = s + 1 + gl + stride * kReg; i < m; i += stride) df_abs2_acc(aj[i], qh, ql);
    const double q2 = warp_sum(f2d_bits(qh) + f2d_bits(ql));
    if (lane == 0) redn[base + wg] = q2;
    group_barrier(1 + grp, 32 * GW);
    t = 0.0;
    for (int k = 0; k < GW; ++k) t += redn[base + k];
    if (gl == 0) *nref_j = t;
  }
  if (gl == 0) aj[s] = top;
  return t;
}

// pv / pi: 2 x gridDim.x partial maxima (parity of the step).  DF: double-float updates
// (the matrix is converted in place after the norm pass and back before the kernel ends).
template <bool DF>
__global__ void __launch_bounds__(kNT, 2) k_pqr(const PqrJob* jobs, int nj, double* pv, int* pi, double tol, int vcap) {
  extern __shared__ cplx sv[];
  __shared__ long long redv[32];
  __shared__ int redi[32];
  __shared__ double redsig[kNT];
  __shared__ cplx redc[2 * kNW];
  __shared__ double redn[2 * kNW];
  __shared__ cplx s_v0;
  __shared__ double s_tau;
  __shared__ dfc s_v0d, s_betad;
  __shared__ float s_th, s_tl;
  int jid = 0;
  while (jid + 1 < nj && jobs[jid + 1].b0 <= (int)blockIdx.x) ++jid;
  const PqrJob jb = jobs[jid];
  const int G = gridDim.x;
  const int lb = (int)blockIdx.x - jb.b0;
  const int64_t m = jb.m, n = jb.n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t gw = (int64_t)lb * kNW + warp, nw = (int64_t)jb.nb * kNW;
  // column groups of GW warps (GW = 1: one warp per column)
  const int GW = jb.gw, grp = warp / GW, wg = warp % GW, gl = wg * 32 + lane;
  const int64_t gg = (int64_t)lb * (kNW / GW) + grp, ngrp = (int64_t)jb.nb * (kNW / GW);
  cplx* A = jb.A;
  dfc* D = reinterpret_cast<dfc*>(jb.A);

  // column norms (FP64) and the first partial maxima (parity 0)
  {
    long long best = kNoKey;
    int bi = 0x7fffffff;
    for (int64_t j = gw; j < n; j += nw) {
      double s2 = 0.0;
      for (int64_t i = lane; i < m; i += 32) {
        const cplx x = A[j * m + i];
        s2 += cabs2(x);
        if constexpr (DF) D[j * m + i] = to_dfc_bits(x);
      }
      s2 = warp_sum(s2);
      if (lane == 0) { jb.nrm[j] = s2; jb.nref[j] = s2; }
      if (better(nkey(s2), (int)j, best, bi)) { best = nkey(s2); bi = (int)j; }
    }
    long long v;
    int ix;
    block_argmax_key<kNT>(best, bi, redv, redi, &v, &ix);
    if (tid == 0) { pv[blockIdx.x] = __longlong_as_double(v); pi[blockIdx.x] = ix; }
  }
  if (group_sync(jb.gs, (unsigned)jb.nb) < 0) return;

  double r00 = 0.0, thr2 = 0.0;
  bool done = false;
  for (int64_t s = 0;; ++s) {
    const int par = (int)(s & 1);
    int p = -1;
    if (!done) {
      long long best = kNoKey;
      int bi = 0x7fffffff;
      for (int q = tid; q < jb.nb; q += kNT) {
        const long long v = nkey(pv[par * G + jb.b0 + q]);
        const int ix = pi[par * G + jb.b0 + q];
        if (better(v, ix, best, bi)) { best = v; bi = ix; }
      }
      long long kmax;
      block_argmax_key<kNT>(best, bi, redv, redi, &kmax, &p);
      const double pvmax = __longlong_as_double(kmax);
      if (s == 0) {
        r00 = sqrt(fmax(pvmax, 0.0));
        thr2 = (tol * r00) * (tol * r00);
      }
      // |R_ss| <= tol |R_00|, compared squared
      const bool tol_met = !(r00 > 0.0) || !(pvmax >= 0.0) || pvmax <= thr2;
      if (tol_met || s >= jb.kcap || s >= m || s >= n || p < 0 || p >= n) {
        done = true;
        if (lb == 0 && tid == 0) {
          jb.st->rank = (int)s;
          jb.st->capped = (!tol_met && s >= jb.kcap && s < m && s < n) ? 1 : 0;
          jb.st->r00 = r00;
        }
      }
    }
    if (!done) {
      const bool staged = (m - s - 1) <= vcap;
      if constexpr (DF) {
        const dfc* ap = D + (int64_t)p * m;
        dfc* svd = reinterpret_cast<dfc*>(sv);
        float qh = 0.f, ql = 0.f;
        for (int64_t i = s + 1 + tid; i < m; i += kNT) {
          const dfc x = ap[i];
          df_abs2_acc(x, qh, ql);
          if (staged) svd[i - s - 1] = x;
        }
        // ||x_{s+1..}||^2 in warp 0, then the reflector by one thread, all in double-float
        // on the FP32 pipes (an FP64 chain costs 64 cycles per instruction here)
        block_sum_df_warp0<kNT>(qh, ql, reinterpret_cast<float*>(redsig));  // also publishes sv
        if (tid == 0) {
          dfc v0, beta;
          float th, tl;
          df_householder(ap[s], qh, ql, &v0, &beta, &th, &tl);
          s_v0d = v0;
          s_betad = beta;
          s_th = th;
          s_tl = tl;
        }
        __syncthreads();
        if (lb == 0 && tid == 32) {  // FP64 copies for the finishing kernels, off the critical path
          jb.piv[s] = p;
          jb.beta[s] = from_dfc_bits(s_betad);
          jb.v0[s] = from_dfc_bits(s_v0d);
          jb.tau[s] = f2d_bits(s_th) + f2d_bits(s_tl);
        }
      } else {
        const cplx* ap = A + (int64_t)p * m;
        double sig = 0.0;
        for (int64_t i = s + 1 + tid; i < m; i += kNT) {
          const cplx x = ap[i];
          sig += cabs2(x);
          if (staged) sv[i - s - 1] = x;
        }
        // The reflector's scalars are formed once per CTA, by lane 0 of warp 0.
        sig = block_sum_warp0<kNT>(sig, redsig);  // also publishes sv to the CTA
        if (tid == 0) {
          cplx v0, beta;
          double tau;
          householder_scalars(ap[s], sig, &v0, &beta, &tau);
          s_v0 = v0;
          s_tau = tau;
          if (lb == 0) {
            jb.piv[s] = p;
            jb.beta[s] = beta;
            jb.v0[s] = v0;
            jb.tau[s] = tau;
          }
        }
        __syncthreads();
      }
      long long best = kNoKey;
      int bi = 0x7fffffff;
      if constexpr (DF) {
        const dfc v0 = s_v0d;
        const float th = s_th, tl = s_tl;
        const dfc* vt = staged ? reinterpret_cast<const dfc*>(sv) : D + (int64_t)p * m + s + 1;
        if (GW == 1) {
          for (int64_t j = gw; j < n; j += nw) {
            const double nj = jb.nrm[j];
            if (nkey(nj) < 0) continue;  // an earlier pivot (marked -1)
            if (j == p) {
              if (lane == 0) jb.nrm[j] = -1.0;
              continue;
            }
            const double t = update_col_warp_df(D + j * m, vt, m, s, v0, th, tl, nj, jb.nref + j, lane);
            if (lane == 0) jb.nrm[j] = t;
            if (better(nkey(t), (int)j, best, bi)) { best = nkey(t); bi = (int)j; }
          }
        } else {
          int slot = 0;
          for (int64_t j = gg; j < n; j += ngrp) {
            const double nj = jb.nrm[j];
            if (nkey(nj) < 0) continue;
            if (j == p) {
              if (gl == 0) jb.nrm[j] = -1.0;
              continue;
            }
            const double t = update_col_group_df(D + j * m, vt, m, s, v0, th, tl, nj, jb.nref + j, gl, GW, grp, wg,
                                                 lane, slot, reinterpret_cast<dfc*>(redc), redn);
            slot ^= 1;
            if (gl == 0) jb.nrm[j] = t;
            if (better(nkey(t), (int)j, best, bi)) { best = nkey(t); bi = (int)j; }
          }
        }
      } else {
        const cplx v0 = s_v0;
        const double tau = s_tau;
        const cplx* vt = staged ? sv : A + (int64_t)p * m + s + 1;
        if (GW == 1) {
          for (int64_t j = gw; j < n; j += nw) {
            const double nj = jb.nrm[j];
            if (nkey(nj) < 0) continue;  // an earlier pivot (marked -1)
            if (j == p) {
              if (lane == 0) jb.nrm[j] = -1.0;
              continue;
            }
            const double t = update_col_warp(A + j * m, vt, m, s, v0, tau, nj, jb.nref + j, lane);
            if (lane == 0) jb.nrm[j] = t;
            if (better(nkey(t), (int)j, best, bi)) { best = nkey(t); bi = (int)j; }
          }
        } else {
          int slot = 0;
          for (int64_t j = gg; j < n; j += ngrp) {
            const double nj = jb.nrm[j];
            if (nkey(nj) < 0) continue;
            if (j == p) {
              if (gl == 0) jb.nrm[j] = -1.0;
              continue;
            }
            const double t = update_col_group(A + j * m, vt, m, s, v0, tau, nj, jb.nref + j, gl, GW, grp, wg, lane,
                                              slot, redc, redn);
            slot ^= 1;
            if (gl == 0) jb.nrm[j] = t;
            if (better(nkey(t), (int)j, best, bi)) { best = nkey(t); bi = (int)j; }
          }
        }
      }
      long long v;
      int ix;
      block_argmax_key<kNT>(best, bi, redv, redi, &v, &ix);
      if (tid == 0) { pv[(1 - par) * G + blockIdx.x] = __longlong_as_double(v); pi[(1 - par) * G + blockIdx.x] = ix; }
    }
    // Every CTA of the matrix takes the same stop decision (the same reduction of the same
    // partial maxima), so all of them leave the loop after the same barrier.
    if (group_sync(jb.gs, (unsigned)jb.nb) < 0 || done) break;
  }
  if constexpr (DF) {
    // Every CTA of this matrix has left the step loop at the same barrier: no update of
    // its columns is in flight.
    for (int64_t j = gw; j < n; j += nw)
      for (int64_t i = lane; i < m; i += 32) A[j * m + i] = from_dfc_bits(D[j * m + i]);
  }
}

// Per matrix (blockIdx.y): the permutation (CTA 0) and R11 as a row-major k x k array
// (all CTAs).  The permutation is the one a column-swapping QR produces (pivot s swapped
// into position s at step s): perm[0..k) = piv, and the other columns in the order those
// swaps leave them.
__global__ void __launch_bounds__(kNT) k_pqr_finish(const PqrJob* jobs) {
  const PqrJob jb = jobs[blockIdx.y];
  const int k = jb.st->rank;
  const int64_t m = jb.m, n = jb.n;
  if (blockIdx.x == 0) {
    for (int64_t i = threadIdx.x; i < n; i += kNT) {
      jb.perm[i] = (int)i;
      jb.pos[i] = (int)i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int s = 0; s < k; ++s) {
        const int p = jb.piv[s], ps = jb.pos[p];
        if (ps != s) {
          const int cs = jb.perm[s];
          jb.perm[s] = p;
          jb.perm[ps] = cs;
          jb.pos[cs] = ps;
          jb.pos[p] = s;
        }
      }
    }
  }
  const int64_t tot = (int64_t)k * k;
  for (int64_t e = blockIdx.x * (int64_t)kNT + threadIdx.x; e < tot; e += (int64_t)gridDim.x * kNT) {
    const int i = (int)(e / k), l = (int)(e % k);
    cplx v = cmk(0.0, 0.0);
    if (l == i) v = jb.beta[i];
    else if (l > i) v = jb.A[(int64_t)jb.piv[l] * m + i];
    jb.r11r[e] = v;
    jb.r11c[(int64_t)l * k + i] = v;
    if (l == i) jb.invd[i] = cdiv(cmk(1.0, 0.0), v);
  }
}

// x = R^{-1} b for upper-triangular R (k <= 32 KR) stored column-major (Rc[i k + r] =
// R(r, i)) with its inverse diagonal, one warp: the column is held in registers (row r in
// lane r % 32, slot r / 32) and x_i is broadcast by shuffle, so the substitution never
// waits on memory.  x is written at the end (it may alias b).
template <int KR>
__device__ __forceinline__ void tsolve_reg_col(const cplx* Rc, const cplx* invd, int k, const cplx* b, cplx* x,
                                               int lane) {
  cplx w[KR];
#pragma unroll
  for (int q = 0; q < KR; ++q) {
    const int r = lane + 32 * q;
    w[q] = r < k ? b[r] : cmk(0.0, 0.0);
  }
#pragma unroll
  for (int qb = KR - 1; qb >= 0; --qb) {
    for (int ii = 31; ii >= 0; --ii) {
      const int i = qb * 32 + ii;
      if (i >= k) continue;
      cplx xi = cmk(__shfl_sync(0xffffffffu, w[qb].x, ii), __shfl_sync(0xffffffffu, w[qb].y, ii));
      xi = cmul(xi, invd[i]);
      if (lane == ii) w[qb] = xi;
      const cplx* ri = Rc + (int64_t)i * k;
#pragma unroll
      for (int q = 0; q <= qb; ++q) {
        const int r = lane + 32 * q;
        if (r < i) w[q] = cfms(ri[r], xi, w[q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < KR; ++q) {
    const int r = lane + 32 * q;
    if (r < k) x[r] = w[q];
  }
}

template <int KR>
__global__ void __launch_bounds__(256) k_tsolve_cols_reg(const cplx* Rc, const cplx* invd, int k, const cplx* B,
                                                         int64_t ldb, int64_t ncols, cplx* X, int64_t ldx) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < ncols; c += nwarps) tsolve_reg_col<KR>(Rc, invd, k, B + c * ldb, X + c * ldx, lane);
}

// The pqr T solves with register-resident columns (every matrix of the batch with k <= 32 KR).
template <int KR>
__global__ void __launch_bounds__(256) k_pqr_tsolve_reg(const PqrJob* jobs) {
  const PqrJob jb = jobs[blockIdx.y];
  const int k = jb.st->rank;
  const int64_t nc = jb.n - k;
  if (k <= 0 || nc <= 0 || jb.T == nullptr) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < nc; c += nwarps)
    tsolve_reg_col<KR>(jb.r11c, jb.invd, k, jb.A + (int64_t)jb.perm[k + c] * jb.m, jb.T + c * (int64_t)k, lane);
}

// Per matrix: T(:, c) = R11^{-1} R12(:, c), R12(:, c) = rows 0..k-1 of physical column
// perm[k + c].  One warp per column.
__global__ void __launch_bounds__(kNT) k_pqr_tsolve(const PqrJob* jobs) {
  const PqrJob jb = jobs[blockIdx.y];
  const int k = jb.st->rank;
  const int64_t nc = jb.n - k;
  if (k <= 0 || nc <= 0 || jb.T == nullptr) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)kNT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kNT) >> 5;
  for (int64_t c = warp; c < nc; c += nwarps) {
    const cplx* b = jb.A + (int64_t)jb.perm[k + c] * jb.m;
    cplx* tc = jb.T + c * (int64_t)k;
    tsolve_row_major(jb.r11r, k, b, tc, lane);
  }
}

}  // namespace

__global__ void __launch_bounds__(256) k_tsolve_cols(const cplx* R, int k, const cplx* B, int64_t ldb, int64_t ncols,
                                                     cplx* X, int64_t ldx) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < ncols; c += nwarps) tsolve_row_major(R, k, B + c * ldb, X + c * ldx, lane);
}

namespace {

// R11 column-major and 1/R_ii from a factorization.
__global__ void k_r11_cols(const cplx* A, int64_t m, const int* piv, const cplx* beta, int k, cplx* Rc, cplx* invd) {
  const int64_t tot = (int64_t)k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % k), i = (int)(e / k);
    cplx v = cmk(0.0, 0.0);
    if (r == i) {
      v = beta[i];
      invd[i] = cdiv(cmk(1.0, 0.0), v);
    } else if (r < i) {
      v = A[(int64_t)piv[i] * m + r];
    }
    Rc[e] = v;
  }
}

// Double-float copy of R11 with its rows scaled by 1/R_ii (column-major, entries r < i), and
// 1/R_ii itself: back substitution then needs no multiply per step,
//   x_i = w'_i,  w'_r -= (R_ri / R_rr) x_i,  with w'_r = b_r / R_rr.
__global__ void k_r11_scaled_df(const cplx* Rc, const cplx* invd, int k, dfc* Rs, dfc* invd_d) {
  const int64_t tot = (int64_t)k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % k), i = (int)(e / k);
    Rs[e] = r < i ? to_dfc_bits(cmul(invd[r], Rc[e])) : dfc{0.f, 0.f, 0.f, 0.f};
    if (i == 0) invd_d[r] = to_dfc_bits(invd[r]);
  }
}

// x = R11^{-1} b for one column per warp, register-resident, in double-float arithmetic.
template <int KR>
__global__ void __launch_bounds__(256) k_tsolve_cols_reg_df(const dfc* Rs, const dfc* invd_d, int k, const cplx* B,
                                                            int64_t ldb, int64_t ncols, cplx* X, int64_t ldx) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < ncols; c += nwarps) {
    const cplx* b = B + c * ldb;
    dfc w[KR];
#pragma unroll
    for (int q = 0; q < KR; ++q) {
      const int r = lane + 32 * q;
      w[q] = r < k ? dfc_mul(to_dfc_bits(b[r]), invd_d[r]) : dfc{0.f, 0.f, 0.f, 0.f};
    }
#pragma unroll
    for (int qb = KR - 1; qb >= 0; --qb) {
      for (int ii = 31; ii >= 0; --ii) {
        const int i = qb * 32 + ii;
        if (i >= k) continue;
        const dfc xi = dfc_shfl(w[qb], ii);
        const dfc* ri = Rs + (int64_t)i * k;
#pragma unroll
        for (int q = 0; q <= qb; ++q) {
          const int r = lane + 32 * q;
          if (r < i) dfc_sub_mul(ri[r], xi, w[q]);
        }
      }
    }
    cplx* x = X + c * ldx;
#pragma unroll
    for (int q = 0; q < KR; ++q) {
      const int r = lane + 32 * q;
      if (r < k) x[r] = from_dfc_bits(w[q]);
    }
  }
}

template <int KR>
void launch_tsolve_reg(const cplx* Rc, const cplx* invd, int k, cplx* W, int64_t ldw, int64_t ncols, cudaStream_t s) {
  if (gemm_double_float()) {
    DevBuf<dfc> Rs((size_t)k * k), inv(k);
    k_r11_scaled_df<<<std::max(1, std::min(4096, (k * k + 255) / 256)), 256, 0, s>>>(Rc, invd, k, Rs.get(), inv.get());
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((ncols + 7) / 8, 152 * 16));
    k_tsolve_cols_reg_df<KR><<<grid, 256, 0, s>>>(Rs.get(), inv.get(), k, W, ldw, ncols, W, ldw);
    return;
  }
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((ncols + 7) / 8, 152 * 16));
  k_tsolve_cols_reg<KR><<<grid, 256, 0, s>>>(Rc, invd, k, W, ldw, ncols, W, ldw);
}

}  // namespace

// W(:, c) <- R11^{-1} W(:, c) for the first k rows, R11 from matrix `job` of a pqr_run.
void pqr_solve_r11(const cplx* A, int64_t m, const PqrOut& qr, int job, int k, cplx* W, int64_t ldw, int64_t ncols,
                   cudaStream_t s) {
  if (k <= 0 || ncols <= 0) return;
  const int* piv = qr.piv.get() + qr.koff[job];
  const cplx* beta = qr.beta.get() + qr.koff[job];
  prof::KScope _ks("k_tsolve_cols", s, 4.0 * k * (double)k * ncols, 0.0);
  if (k <= 512) {
    DevBuf<cplx> Rc((size_t)k * k), invd(k);
    k_r11_cols<<<std::max(1, std::min(4096, (k * k + 255) / 256)), 256, 0, s>>>(A, m, piv, beta, k, Rc.get(),
                                                                                 invd.get());
    switch ((k + 31) / 32) {
      case 1: launch_tsolve_reg<1>(Rc.get(), invd.get(), k, W, ldw, ncols, s); break;
      case 2: launch_tsolve_reg<2>(Rc.get(), invd.get(), k, W, ldw, ncols, s); break;
      case 3: launch_tsolve_reg<3>(Rc.get(), invd.get(), k, W, ldw, ncols, s); break;
      case 4: launch_tsolve_reg<4>(Rc.get(), invd.get(), k, W, ldw, ncols, s); break;
      case 5: launch_tsolve_reg<5>(Rc.get(), invd.get(), k, W, ldw, ncols, s); break;
      case 6: launch_tsolve_reg<6>(Rc.get(), invd.get(), k, W, ldw, ncols, s); break;
      case 7: launch_tsolve_reg<7>(Rc.get(), invd.get(), k, W, ldw, ncols, s); break;
      case 8: launch_tsolve_reg<8>(Rc.get(), invd.get(), k, W, ldw, ncols, s); break;
      case 9: case 10: case 11: case 12: launch_tsolve_reg<12>(Rc.get(), invd.get(), k, W, ldw, ncols, s); break;
      default: launch_tsolve_reg<16>(Rc.get(), invd.get(), k, W, ldw, ncols, s); break;
    }
  } else {
    DevBuf<cplx> R((size_t)k * k);
    k_r11_rows<<<std::max(1, std::min(4096, (k * k + 255) / 256)), 256, 0, s>>>(A, m, piv, beta, k, R.get());
    k_tsolve_cols<<<(int)std::max<int64_t>(1, std::min<int64_t>((ncols + 7) / 8, 4096)), 256, 0, s>>>(
        R.get(), k, W, ldw, ncols, W, ldw);
  }
  HBS_LAUNCH_CHECK("pqr_solve_r11");
}

// Column j of conj(Q1) (Q1 = first k columns of H_0 ... H_{k-1}):  q = H_0 ... H_j e_j.
// One CTA per column; q lives in the output column.
__global__ void __launch_bounds__(kNT) k_form_qc(const cplx* A, int64_t m, const int* piv, const cplx* v0,
                                                 const double* tau, int k, cplx* Qc) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  if (j >= k) return;
  cplx* q = Qc + (int64_t)j * m;
  for (int64_t i = threadIdx.x; i < m; i += kNT) q[i] = cmk(i == j ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int s = j; s >= 0; --s) {
    const cplx* ap = A + (int64_t)piv[s] * m;
    const cplx h0 = v0[s];
    cplx w = cmk(0.0, 0.0);
    if (threadIdx.x == 0) w = cmul(cconj(h0), q[s]);
    for (int64_t i = s + 1 + threadIdx.x; i < m; i += kNT) w = cfma(cconj(ap[i]), q[i], w);
    w = block_sum_c<kNT>(w, red);
    w = cscale(w, tau[s]);
    if (threadIdx.x == 0) q[s] = cfms(h0, w, q[s]);
    for (int64_t i = s + 1 + threadIdx.x; i < m; i += kNT) q[i] = cfms(ap[i], w, q[i]);
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < m; i += kNT) q[i] = cconj(q[i]);
}

// R11 (k x k, row-major) from the factored matrix.
__global__ void k_r11_rows(const cplx* A, int64_t m, const int* piv, const cplx* beta, int k, cplx* R) {
  const int64_t tot = (int64_t)k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), l = (int)(e % k);
    cplx v = cmk(0.0, 0.0);
    if (l == i) v = beta[i];
    else if (l > i) v = A[(int64_t)piv[l] * m + i];
    R[e] = v;
  }
}

// out[r + c ldo] = src[r + idx[c] lds]: columns idx of src.
__global__ void k_gather_cols(const cplx* src, int64_t lds, int64_t rows, const int64_t* idx, int64_t ncols, cplx* out,
                              int64_t ldo) {
  const int64_t tot = rows * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows, c = e / rows;
    out[r + c * ldo] = src[r + idx[c] * lds];
  }
}

// X(:, idx[c]) = e_c for c < k (X: k x ncols, ld k).
__global__ void k_set_unit_cols(cplx* X, int k, const int64_t* idx) {
  const int64_t tot = (int64_t)k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % k), c = (int)(e / k);
    X[r + idx[c] * (int64_t)k] = cmk(r == c ? 1.0 : 0.0, 0.0);
  }
}

// Warps per column group for a matrix on b CTAs: doubled while the groups still cover
// every column and each lane keeps at least four rows.
static int col_group_warps(int b, int64_t m, int64_t n) {
  int g = 1;
  while (g < 8 && (int64_t)b * (kNW / (2 * g)) >= n && m >= (int64_t)32 * (2 * g) * 4) g *= 2;
  return g;
}

template <bool DF>
static int pqr_grid(size_t smem) {
  static const int sms = [] {
    int dev = 0, sm = 0;
    HBS_CUDA(cudaGetDevice(&dev));
    HBS_CUDA(cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev));
    return sm;
  }();
  HBS_CUDA(raise_smem_limit((const void*)k_pqr<DF>, smem));
  int per_sm = 0;
  HBS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pqr<DF>, kNT, smem));
  if (per_sm < 1) throw Error(HBS_ERR_CUDA, "persistent QR kernel does not fit on an SM");
  return sms * std::min(per_sm, background_chain() ? 1 : 2);
}

void pqr_run(const std::vector<PqrSpec>& specs_in, double tol, cudaStream_t s, PqrOut& out, bool equal_steps) {
  // a rank cap set by hbs_fault_inject (tests of the HBS_ERR_RANK path) lowers every kcap
  std::vector<PqrSpec> specs(specs_in);
  if (const int cap = injected_rank_cap(); cap > 0)
    for (auto& sp : specs) sp.kcap = std::min(sp.kcap, cap);
  const int nj = (int)specs.size();
  out.rank.assign(nj, 0);
  out.koff.assign(nj + 1, 0);
  if (nj == 0) return;
  int64_t mmax = 0, ntot = 0;
  for (int j = 0; j < nj; ++j) {
    const auto& sp = specs[j];
    mmax = std::max(mmax, sp.m);
    ntot += sp.n;
    out.koff[j + 1] = out.koff[j] + std::max(1, sp.kcap);
  }
  const int vcap = (int)std::min<int64_t>(mmax, 6144);
  const size_t smem = (size_t)vcap * sizeof(cplx);
  // Double-float updates on handles built with double-float precision; the public row ID
  // entry points keep FP64 throughout.
  const bool df = gemm_double_float();
  const int G = df ? pqr_grid<true>(smem) : pqr_grid<false>(smem);
  if (nj > G) throw Error(HBS_ERR_INTERNAL, "persistent QR batch larger than the grid");
  // CTAs per matrix: a step of matrix j on b CTAs takes about as long as its busiest
  // column group's work (columns per group x rows per lane, the groups' width GW as chosen
  // below) plus a fixed cost of the pivot choice, the reflector and the barrier (about 24
  // such units, measured), for up to min(m, n, kcap) steps (or the same number for all).
  const std::vector<int> nb = balance_ctas(G, nj, [&](int j, int b) {
    const auto& sp = specs[j];
    const int g = col_group_warps(b, sp.m, sp.n);
    const int64_t groups = (int64_t)b * (kNW / g);
    const double cols = (double)((sp.n + groups - 1) / groups);
    const double rows = (double)((sp.m + 32 * g - 1) / (32 * g));
    const double steps =
        equal_steps ? 1.0 : (double)std::max<int64_t>(1, std::min<int64_t>(sp.kcap, std::min(sp.m, sp.n)));
    return steps * (cols * rows + 24.0);
  });
  const int64_t ktot = out.koff[nj];
  int64_t r11tot = 0;
  std::vector<int64_t> r11off(nj);
  for (int j = 0; j < nj; ++j) {
    r11off[j] = r11tot;
    const int64_t kk = std::min<int64_t>(specs[j].kcap, std::min(specs[j].m, specs[j].n));
    r11tot += kk * kk;
  }
  DevBuf<double> nrm(ntot), nref(ntot), pv(2 * (size_t)G);
  DevBuf<int> pi(2 * (size_t)G), pos(ntot);
  out.piv.alloc(ktot);
  out.beta.alloc(ktot);
  out.v0.alloc(ktot);
  out.tau.alloc(ktot);
  DevBuf<PqrState> st(nj);
  DevBuf<GridSync> gs(nj);
  DevBuf<cplx> r11(std::max<int64_t>(r11tot, 1)), r11c(std::max<int64_t>(r11tot, 1)), invd(std::max<int64_t>(ktot, 1));
  HBS_CUDA(cudaMemsetAsync(st.get(), 0, sizeof(PqrState) * nj, s));
  HBS_CUDA(cudaMemsetAsync(gs.get(), 0, sizeof(GridSync) * nj, s));
  std::vector<PqrJob> jobs(nj);
  int64_t o = 0;
  int b0 = 0;
  for (int j = 0; j < nj; ++j) {
    const auto& sp = specs[j];
    const int gwv = col_group_warps(nb[j], sp.m, sp.n);
    jobs[j] = {sp.A, sp.m, sp.n, sp.kcap, b0, nb[j], gwv, nrm.get() + o, nref.get() + o,
               out.piv.get() + out.koff[j], out.beta.get() + out.koff[j], out.v0.get() + out.koff[j],
               out.tau.get() + out.koff[j], st.get() + j, sp.perm, sp.T, r11.get() + r11off[j],
               r11c.get() + r11off[j], invd.get() + out.koff[j], pos.get() + o, gs.get() + j};
    o += sp.n;
    b0 += nb[j];
  }
  DevBuf<PqrJob> dj;
  dj.upload(jobs, s);
  const PqrJob* a0 = dj.get();
  int a1 = nj;
  double* a2 = pv.get();
  int* a3 = pi.get();
  double a5 = tol;
  int a6 = vcap;
  void* args[] = {&a0, &a1, &a2, &a3, &a5, &a6};
  std::vector<PqrState> hs(nj);
  std::vector<GridSync> hg(nj);
  {
    std::lock_guard<std::mutex> lock(coop_mutex());
    {
      prof::KScope _ks("k_pqr", s);
      const void* fn = df ? (const void*)k_pqr<true> : (const void*)k_pqr<false>;
      HBS_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kNT), args, smem, s));
    }
    HBS_LAUNCH_CHECK("k_pqr");
    read_to_host(hs.data(), st.get(), sizeof(PqrState) * nj, s);
    read_to_host(hg.data(), gs.get(), sizeof(GridSync) * nj, s);
  }
  for (const auto& g : hg)
    if (g.timed_out) throw Error(HBS_ERR_TIMEOUT, "persistent QR: a barrier wait gave up");
  int kmax = 0;
  int64_t nmax = 0;
  for (int j = 0; j < nj; ++j) {
    out.rank[j] = hs[j].rank;
    if (hs[j].capped) throw Error(HBS_ERR_RANK, "interpolative decomposition rank exceeds the supported maximum");
    kmax = std::max(kmax, hs[j].rank);
    nmax = std::max(nmax, specs[j].n);
  }
  {
    prof::KScope _ks("k_pqr_finish", s);
    k_pqr_finish<<<dim3(8, nj), kNT, 0, s>>>(dj.get());
  }
  {
    prof::KScope _ks("k_pqr_tsolve", s);
    const int bx = (int)std::max<int64_t>(1, std::min<int64_t>(1216 / nj + 1, (nmax + kNW - 1) / kNW));
    const dim3 grid(bx, nj);
    switch ((kmax + 31) / 32) {
      case 0:
      case 1: k_pqr_tsolve_reg<1><<<grid, 256, 0, s>>>(dj.get()); break;
      case 2: k_pqr_tsolve_reg<2><<<grid, 256, 0, s>>>(dj.get()); break;
      case 3: k_pqr_tsolve_reg<3><<<grid, 256, 0, s>>>(dj.get()); break;
      case 4: k_pqr_tsolve_reg<4><<<grid, 256, 0, s>>>(dj.get()); break;
      case 5: k_pqr_tsolve_reg<5><<<grid, 256, 0, s>>>(dj.get()); break;
      case 6: k_pqr_tsolve_reg<6><<<grid, 256, 0, s>>>(dj.get()); break;
      case 7: k_pqr_tsolve_reg<7><<<grid, 256, 0, s>>>(dj.get()); break;
      case 8: k_pqr_tsolve_reg<8><<<grid, 256, 0, s>>>(dj.get()); break;
      case 9: case 10: case 11: case 12: k_pqr_tsolve_reg<12><<<grid, 256, 0, s>>>(dj.get()); break;
      case 13: case 14: case 15: case 16: k_pqr_tsolve_reg<16><<<grid, 256, 0, s>>>(dj.get()); break;
      default: k_pqr_tsolve<<<grid, kNT, 0, s>>>(dj.get()); break;
    }
  }
  HBS_LAUNCH_CHECK("k_pqr_finish");
  // algorithmic work of an interpolative decomposition of an m x n block of rank k: 8 m n k
  // flops (the Householder factorization executes about twice that), and the block read
  // once plus the interpolation matrix and the order written once
  double fl = 0.0, by = 0.0;
  for (int j = 0; j < nj; ++j) {
    const double m = (double)specs[j].m, n = (double)specs[j].n, k = out.rank[j];
    fl += 8.0 * m * n * k;
    by += 16.0 * m * n + 16.0 * k * (n - k) + 4.0 * n;
  }
  prof::add_work("k_pqr", fl, by);
}

}  // namespace hbs
