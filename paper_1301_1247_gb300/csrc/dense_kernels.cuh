// Batched small dense complex FP64 kernels used by the HBS build (Sec. 4):
// column-pivoted QR for the interpolative decomposition (Def. 3.1) and
// Gauss-Jordan inversion with partial pivoting for the per-node blocks.
// One CTA works on one matrix; matrices live in global memory (L2-resident).
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace hbs {

// Descriptor of one matrix of a batch (pointers into any device buffers, so a batch may
// span several solvers).
struct CpqrJob {
  cplx* mt;    // Mt (m x n, ld = m), overwritten
  cplx* t;     // T output (k x (n - k), ld = k; capacity min(m,n) * n)
  int* perm;   // perm output (n ints)
  int m, n;
  int job;     // index into the rank output array
};

struct InvJob {
  cplx* a;     // matrix (n x n, ld = n), inverted in place
  int* piv;    // int scratch (n), set by the launcher
  int n;
  int job;
};

// Block-wide reduction helpers (NT threads, NT multiple of 32).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

// Sum over the block formed in warp 0 alone, so that the other warps issue no FP64
// instructions for it: the values meet in shared memory (red: NT doubles), lane l of
// warp 0 adds those of threads l, l + 32, ... and a butterfly finishes.  The sum is
// returned in every lane of warp 0 (other threads get an unspecified value).  Contains
// one __syncthreads; red may be reused after the caller's next barrier.
template <int NT>
__device__ __forceinline__ double block_sum_warp0(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) t += red[threadIdx.x + 32 * k];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

// Householder reflector H = I - tau v v^H with v = (v0, x_1, x_2, ...) mapping
// x = (x0, x_1, ...) to (beta, 0, ...), beta = -(x0/|x0|) ||x|| (sig = sum_{i>0} |x_i|^2).
__device__ __forceinline__ void householder_scalars(cplx x0, double sig, cplx* v0, cplx* beta, double* tau) {
  const double ax0 = cabs1(x0);
  const double xn = sqrt(ax0 * ax0 + sig);
  const cplx ph = ax0 > 0.0 ? cmk(x0.x / ax0, x0.y / ax0) : cmk(1.0, 0.0);
  *beta = cmk(-ph.x * xn, -ph.y * xn);
  *v0 = csub(x0, *beta);
  const double vv = cabs2(*v0) + sig;
  *tau = vv > 0.0 ? 2.0 / vv : 0.0;
}

// Pivot searches compare squared moduli as IEEE-754 bit patterns read as signed 64-bit
// integers: for non-negative doubles the order is the same, and a -1 marker (an
// eliminated column) sorts below all of them, so the search takes exactly the decisions
// of a floating-point search while leaving the FP64 pipe (1/64 of the FP32 rate on
// GB300; its instructions cost the same with one active lane as with 32) to the updates.
__device__ __forceinline__ long long nkey(double v) { return __double_as_longlong(v); }

__device__ __forceinline__ bool better(long long v, int i, long long bv, int bi) {
  return v > bv || (v == bv && i < bi);
}

constexpr long long kNoKey = (long long)0xBFF0000000000000ull;  // bits of -1.0

// Block-wide (key, index) maximum, lowest index on ties, in every thread.
template <int NT>
__device__ __forceinline__ void block_argmax_key(long long v, int idx, long long* redv, int* redi, long long* outv,
                                                 int* outi) {
  for (int o = 16; o > 0; o >>= 1) {
    const long long v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (better(v2, i2, v, idx)) { v = v2; idx = i2; }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { redv[warp] = v; redi[warp] = idx; }
  __syncthreads();
  if (threadIdx.x < 32) {
    long long t = threadIdx.x < NT / 32 ? redv[threadIdx.x] : kNoKey;
    int ti = threadIdx.x < NT / 32 ? redi[threadIdx.x] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      const long long t2 = __shfl_xor_sync(0xffffffffu, t, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, ti, o);
      if (better(t2, i2, t, ti)) { t = t2; ti = i2; }
    }
    if (threadIdx.x == 0) { redv[0] = t; redi[0] = ti; }
  }
  __syncthreads();
  *outv = redv[0];
  *outi = redi[0];
  __syncthreads();
}

// Returns (max value, lowest index attaining it) over the block.
template <int NT>
__device__ __forceinline__ void block_argmax(double v, int idx, double* redv, int* redi, double* outv,
                                             int* outi) {
  for (int o = 16; o > 0; o >>= 1) {
    double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (v2 > v || (v2 == v && i2 < idx)) { v = v2; idx = i2; }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { redv[warp] = v; redi[warp] = idx; }
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < NT / 32 ? redv[threadIdx.x] : -1.0;
    int ti = threadIdx.x < NT / 32 ? redi[threadIdx.x] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      double t2 = __shfl_xor_sync(0xffffffffu, t, o);
      int i2 = __shfl_xor_sync(0xffffffffu, ti, o);
      if (t2 > t || (t2 == t && i2 < ti)) { t = t2; ti = i2; }
    }
    if (threadIdx.x == 0) { redv[0] = t; redi[0] = ti; }
  }
  __syncthreads();
  *outv = redv[0];
  *outi = redi[0];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Column-pivoted Householder QR of Mt (m x n) with rank revealed at
// |R_ss| <= tol |R_00| (the interpolative decomposition of Def. 3.1 applied to
// the rows of M = Mt^T).  Column norms are downdated after each reflection
// and recomputed when cancellation has removed more than 7/8 of their digits
// (relative to the norm at the last recomputation).
// Dynamic shared memory: 2 n doubles + n ints.
// ---------------------------------------------------------------------------
// DF: the matrix is held in place as complex double-float (dfc) between the norm pass
// and the triangular solve, and the rank-one updates run in double-float arithmetic on
// the FP32 pipes; norms, pivots and the reflector scalars stay FP64.
template <int NT, bool DF>
__global__ void __launch_bounds__(NT) k_cpqr(const CpqrJob* jobs, int* rank_out, double tol, int kmax) {
  extern __shared__ double smem[];
  __shared__ long long redv[32];
  __shared__ int redi[32];
  __shared__ double redsig[NT];
  __shared__ cplx sh_v0;
  __shared__ double sh_tau;
  __shared__ dfc sh_v0d;
  __shared__ float sh_th, sh_tl;

  const CpqrJob jb = jobs[blockIdx.x];
  const int m = jb.m, n = jb.n;
  cplx* A = jb.mt;
  double* nrm = smem;          // current squared norms of the trailing parts
  double* nrm_ref = smem + n;  // reference norms for the cancellation test
  int* perm = reinterpret_cast<int*>(smem + 2 * n);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;

  dfc* D = reinterpret_cast<dfc*>(A);
  // initial column norms (one warp per column)
  for (int j = warp; j < n; j += NW) {
    double s = 0.0;
    cplx* col = A + (int64_t)j * m;
    for (int i = lane; i < m; i += 32) {
      const cplx x = col[i];
      s += cabs2(x);
      if constexpr (DF) reinterpret_cast<dfc*>(col)[i] = to_dfc_bits(x);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) { nrm[j] = s; nrm_ref[j] = s; }
  }
  for (int j = tid; j < n; j += NT) perm[j] = j;
  __syncthreads();

  const int kcap = min(min(m, n), kmax);
  double r00 = 0.0, thr2 = 0.0;
  int rank = 0;
  for (int s = 0; s < kcap; ++s) {
    long long best = kNoKey;
    int bi = 0x7fffffff;
    for (int j = s + tid; j < n; j += NT) {
      const long long v = nkey(nrm[j]);
      if (better(v, j, best, bi)) { best = v; bi = j; }
    }
    long long kv;
    int p;
    block_argmax_key<NT>(best, bi, redv, redi, &kv, &p);
    const double pv = __longlong_as_double(kv);
    if (s == 0) {
      r00 = sqrt(pv);
      thr2 = (tol * r00) * (tol * r00);
    }
    // |R_ss| <= tol |R_00|, compared squared
    if (!(r00 > 0.0) || !(pv >= 0.0) || pv <= thr2) break;
    // swap columns s and p
    if (p != s) {
      cplx* cs = A + (int64_t)s * m;
      cplx* cp = A + (int64_t)p * m;
      for (int i = tid; i < m; i += NT) { cplx t = cs[i]; cs[i] = cp[i]; cp[i] = t; }
      if (tid == 0) {
        double t = nrm[s]; nrm[s] = nrm[p]; nrm[p] = t;
        t = nrm_ref[s]; nrm_ref[s] = nrm_ref[p]; nrm_ref[p] = t;
        int ti = perm[s]; perm[s] = perm[p]; perm[p] = ti;
      }
    }
    __syncthreads();
    if constexpr (DF) {
      // Householder reflector for x = A[s:m, s]
      dfc* cs = D + (int64_t)s * m;
      float qh = 0.f, ql = 0.f;
      for (int i = s + 1 + tid; i < m; i += NT) df_abs2_acc(cs[i], qh, ql);
      const double sig = block_sum_warp0<NT>(f2d_bits(qh) + f2d_bits(ql), redsig);
      if (tid == 0) {
        cplx v0, beta;
        double tau;
        householder_scalars(from_dfc_bits(cs[s]), sig, &v0, &beta, &tau);
        sh_v0d = to_dfc_bits(v0);
        float th, tl;
        df_split_bits(tau, th, tl);
        sh_th = th;
        sh_tl = tl;
        cs[s] = to_dfc_bits(beta);  // R_ss
      }
      __syncthreads();
      const dfc v0 = sh_v0d;
      const float th = sh_th, tl = sh_tl;
      for (int j = s + 1 + warp; j < n; j += NW) {
        dfc* cj = D + (int64_t)j * m;
        dfc w = {0.f, 0.f, 0.f, 0.f};
        for (int i = s + 1 + lane; i < m; i += 32) dfc_cdot_acc(cs[i], cj[i], w);
        w = dfc_warp_sum(w);
        const dfc ajs = cj[s];
        dfc_cdot_acc(v0, ajs, w);
        dfc_norm(w);
        const dfc wv = dfc_scale(th, tl, w);
        for (int i = s + 1 + lane; i < m; i += 32) {
          dfc a = cj[i];
          dfc_sub_mul(cs[i], wv, a);
          cj[i] = a;
        }
        dfc top = ajs;
        dfc_sub_mul(v0, wv, top);
        __syncwarp();
        // norm downdate, recomputation on cancellation (uniform over the warp)
        float ph = 0.f, pl = 0.f;
        df_abs2_acc(top, ph, pl);
        double t = (nrm[j] - f2d_bits(ph)) - f2d_bits(pl);
        if (t <= 0.0078125 * nrm_ref[j]) {
          float rh = 0.f, rl = 0.f;
          for (int i = s + 1 + lane; i < m; i += 32) df_abs2_acc(cj[i], rh, rl);
          double q = f2d_bits(rh) + f2d_bits(rl);
          for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
          t = q;
          if (lane == 0) nrm_ref[j] = t;
        }
        __syncwarp();
        if (lane == 0) {
          cj[s] = top;
          nrm[j] = t;
        }
      }
      __syncthreads();
      rank = s + 1;
      continue;
    }
    // Householder reflector for x = A[s:m, s]
    cplx* cs = A + (int64_t)s * m;
    double sig = 0.0;
    for (int i = s + 1 + tid; i < m; i += NT) sig += cabs2(cs[i]);
    sig = block_sum_warp0<NT>(sig, redsig);
    if (tid == 0) {
      cplx v0, beta;
      double tau;
      householder_scalars(cs[s], sig, &v0, &beta, &tau);
      sh_v0 = v0;
      sh_tau = tau;
      cs[s] = beta;  // R_ss
    }
    __syncthreads();
    const cplx v0 = sh_v0;
    const double tau = sh_tau;
    // apply H = I - tau v v^H to columns s+1..n-1 (one warp per column)
    for (int j = s + 1 + warp; j < n; j += NW) {
      cplx* cj = A + (int64_t)j * m;
      cplx w = cmk(0.0, 0.0);
      for (int i = s + 1 + lane; i < m; i += 32) w = cfma(cconj(cs[i]), cj[i], w);
      for (int o = 16; o > 0; o >>= 1) {
        w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
        w.y += __shfl_xor_sync(0xffffffffu, w.y, o);
      }
      w = cfma(cconj(v0), cj[s], w);
      w = cscale(w, tau);
      if (lane == 0) cj[s] = cfms(v0, w, cj[s]);
      for (int i = s + 1 + lane; i < m; i += 32) cj[i] = cfms(cs[i], w, cj[i]);
      __syncwarp();
      // norm downdate, recomputation on cancellation
      if (lane == 0) {
        double t = nrm[j] - cabs2(cj[s]);
        nrm[j] = t;
      }
      __syncwarp();
      if (nrm[j] <= 0.0078125 * nrm_ref[j]) {
        double t = 0.0;
        for (int i = s + 1 + lane; i < m; i += 32) t += cabs2(cj[i]);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) { nrm[j] = t; nrm_ref[j] = t; }
      }
    }
    __syncthreads();
    rank = s + 1;
  }
  // T = R11^{-1} R12, one warp per column of R12
  const int k = rank;
  if constexpr (DF) {
    // back to FP64: rows < k of every column (R11, R12; the rest is scratch)
    __syncthreads();
    for (int j = warp; j < n; j += NW)
      for (int i = lane; i < min(k, m); i += 32) A[(int64_t)j * m + i] = from_dfc_bits(D[(int64_t)j * m + i]);
    __syncthreads();
  }
  cplx* T = jb.t;
  for (int c = warp; c < n - k; c += NW) {
    const cplx* r12 = A + (int64_t)(k + c) * m;
    cplx* tc = T + (int64_t)c * k;
    for (int i = k - 1; i >= 0; --i) {
      cplx acc = cmk(0.0, 0.0);
      for (int l = i + 1 + lane; l < k; l += 32) acc = cfma(A[(int64_t)l * m + i], tc[l], acc);
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) tc[i] = cdiv(csub(r12[i], acc), A[(int64_t)i * m + i]);
      __syncwarp();
    }
  }
  int* po = jb.perm;
  for (int j = tid; j < n; j += NT) po[j] = perm[j];
  if (tid == 0) rank_out[jb.job] = k;
}

// ---------------------------------------------------------------------------
// In-place inverse of an n x n matrix by Gauss-Jordan elimination with
// partial (row) pivoting; column interchanges are undone at the end.
// rank_out[job] receives 0 on success, or 1 if a zero pivot was met.
// ---------------------------------------------------------------------------
// DF: the block is held in place as complex double-float between a conversion at the start
// and one at the end, and the eliminations run in double-float arithmetic on the FP32
// pipes; pivots are chosen on |a|^2 to float precision.
template <int NT, bool DF>
__global__ void __launch_bounds__(NT) k_gj_inverse(const InvJob* jobs, int* flag_out) {
  __shared__ long long redv[32];
  __shared__ int redi[32];
  __shared__ cplx sh_piv;
  __shared__ dfc sh_pivd;
  const InvJob jb = jobs[blockIdx.x];
  const int n = jb.n;
  cplx* A = jb.a;
  dfc* D = reinterpret_cast<dfc*>(jb.a);
  int* piv = jb.piv;
  const int tid = threadIdx.x;
  int bad = 0;
  if constexpr (DF) {
    for (int64_t e = tid; e < (int64_t)n * n; e += NT) D[e] = to_dfc_bits(A[e]);
    __syncthreads();
  }
  for (int c = 0; c < n; ++c) {
    long long best = kNoKey;
    int bi = 0x7fffffff;
    for (int i = c + tid; i < n; i += NT) {
      long long v;
      if constexpr (DF) {
        const dfc x = D[(int64_t)c * n + i];
        v = (long long)__float_as_uint(fmaf(x.rh, x.rh, x.ih * x.ih));
      } else {
        v = nkey(cabs2(A[(int64_t)c * n + i]));
      }
      if (better(v, i, best, bi)) { best = v; bi = i; }
    }
    long long kv;
    int p;
    block_argmax_key<NT>(best, bi, redv, redi, &kv, &p);
    const bool nonzero = DF ? (__uint_as_float((unsigned int)kv) > 0.f) : (__longlong_as_double(kv) > 0.0);
    if (tid == 0) piv[c] = p;
    if (!nonzero) { bad = 1; p = c; }
    if constexpr (DF) {
      if (p != c) {
        for (int j = tid; j < n; j += NT) {
          const dfc t = D[(int64_t)j * n + c];
          D[(int64_t)j * n + c] = D[(int64_t)j * n + p];
          D[(int64_t)j * n + p] = t;
        }
      }
      __syncthreads();
      if (tid == 0) sh_pivd = dfc_recip(D[(int64_t)c * n + c]);
      __syncthreads();
      const dfc ip = sh_pivd;
      // scale pivot row: A[c, :] *= 1/d, with A[c,c] := 1/d
      for (int j = tid; j < n; j += NT) {
        if (j == c) D[(int64_t)c * n + c] = ip;
        else D[(int64_t)j * n + c] = dfc_mul(D[(int64_t)j * n + c], ip);
      }
      __syncthreads();
      // eliminate: for rows i != c: A[i, j] -= A[i, c] * A[c, j]  (j != c)
      for (int64_t e = tid; e < (int64_t)n * n; e += NT) {
        const int i = (int)(e % n), j = (int)(e / n);
        if (i == c || j == c) continue;
        dfc x = D[(int64_t)j * n + i];
        dfc_sub_mul(D[(int64_t)c * n + i], D[(int64_t)j * n + c], x);
        D[(int64_t)j * n + i] = x;
      }
      __syncthreads();
      for (int i = tid; i < n; i += NT) {
        if (i != c) {
          const dfc t = dfc_mul(D[(int64_t)c * n + i], ip);
          D[(int64_t)c * n + i] = {-t.rh, -t.rl, -t.ih, -t.il};
        }
      }
      __syncthreads();
    } else {
      if (p != c) {
        for (int j = tid; j < n; j += NT) {
          cplx t = A[(int64_t)j * n + c];
          A[(int64_t)j * n + c] = A[(int64_t)j * n + p];
          A[(int64_t)j * n + p] = t;
        }
      }
      __syncthreads();
      if (tid == 0) {
        cplx d = A[(int64_t)c * n + c];
        sh_piv = (cabs2(d) > 0.0) ? cdiv(cmk(1.0, 0.0), d) : cmk(0.0, 0.0);
      }
      __syncthreads();
      const cplx ip = sh_piv;
      // scale pivot row: A[c, :] *= 1/d, with A[c,c] := 1/d
      for (int j = tid; j < n; j += NT) {
        if (j == c) A[(int64_t)c * n + c] = ip;
        else A[(int64_t)j * n + c] = cmul(A[(int64_t)j * n + c], ip);
      }
      __syncthreads();
      // eliminate: for rows i != c: A[i, j] -= A[i, c] * A[c, j]  (j != c); A[i, c] = -A[i, c] / d
      for (int64_t e = tid; e < (int64_t)n * n; e += NT) {
        int i = (int)(e % n), j = (int)(e / n);
        if (i == c || j == c) continue;
        A[(int64_t)j * n + i] = cfms(A[(int64_t)c * n + i], A[(int64_t)j * n + c], A[(int64_t)j * n + i]);
      }
      __syncthreads();
      for (int i = tid; i < n; i += NT) {
        if (i != c) A[(int64_t)c * n + i] = cmul(cmk(-A[(int64_t)c * n + i].x, -A[(int64_t)c * n + i].y), ip);
      }
      __syncthreads();
    }
  }
  if constexpr (DF) {
    for (int64_t e = tid; e < (int64_t)n * n; e += NT) A[e] = from_dfc_bits(D[e]);
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, in reverse order
  for (int c = n - 1; c >= 0; --c) {
    int p = piv[c];
    if (p != c) {
      for (int i = tid; i < n; i += NT) {
        cplx t = A[(int64_t)c * n + i];
        A[(int64_t)c * n + i] = A[(int64_t)p * n + i];
        A[(int64_t)p * n + i] = t;
      }
    }
    __syncthreads();
  }
  if (tid == 0) flag_out[jb.job] = bad;
}

}  // namespace hbs
