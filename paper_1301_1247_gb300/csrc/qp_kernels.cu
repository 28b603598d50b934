// Periodizing blocks and neighbour images on the device (Secs. 2.2-2.4, 3.2):
// Sommerfeld-contour wall potentials B_L, B_R (Eqs. Sh, Dh, B), Fourier wall rows
// C_L, C_R (operators S^, D^, D*^, T^ and Eq. C with the image reading of Sec. 2.4),
// Bragg sampling rows (Remarks 2.2, 2.3), the neighbour interpolative decomposition
// (Sec. 3.2) as a multi-CTA column-pivoted QR over all N boundary points.
#include "dense_kernels.cuh"
#include "profile.hpp"
#include "handle.hpp"
#include "qp_kernels.cuh"

namespace hbs {

__device__ __forceinline__ cplx sqrt_branch(double omega, cplx k) {
  // sqrt(omega - k) * sqrt(omega + k), principal roots (cuts on the real axis beyond +-omega)
  return cmul(csqrt_principal(cmk(omega - k.x, -k.y)), csqrt_principal(cmk(omega + k.x, k.y)));
}

// Transmission sigma rows of the wall potentials: minus the normal derivative of
// e^{i k y} e^{i s |x - x0|} over w, i.e. the value times -i (+-s n_x + k n_y) / w (+ for
// the left wall, x > x0; - for the right wall).
__device__ __forceinline__ cplx wall_sigma_factor(const DevGeom& g, int64_t i, cplx s, cplx km, bool left) {
  const double sx = left ? g.nx[i] : -g.nx[i];
  const cplx a = cscale(cadd(cscale(s, sx), cscale(km, g.ny[i])), 1.0 / g.omega);
  return cmk(a.y, -a.x);
}

// B_L and B_R columns (N x 2M each) for one contour, written into W (ld = N) at
// columns [col_bl, col_bl + 2M) and [col_br, col_br + 2M).  Optionally combined as
// B_L + alpha B_R into col_bl only (alpha_only != 0).
__global__ void k_fill_b(DevGeom g, const cplx* k, const cplx* wk, int M, double d, cplx* W, int64_t ldw,
                         int64_t col_bl, int64_t col_br, int combine, cplx alpha) {
  const int64_t tot = g.n * (int64_t)M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % g.n;
    const int m = (int)(e / g.n);
    const cplx km = k[m], w = wk[m];
    const cplx s = sqrt_branch(g.omega, km);
    const double xi = g.x[i], yi = g.y[i];
    // e^{i k y} e^{i s |x - x0|} for x0 = -d/2 (L) and x0 = d/2 (R)
    cplx eky = cexp(cmk(-km.y * yi, km.x * yi));
    double al = xi + 0.5 * d, ar = 0.5 * d - xi;
    cplx el = cmul(eky, cexp(cmk(-s.y * al, s.x * al)));
    cplx er = cmul(eky, cexp(cmk(-s.y * ar, s.x * ar)));
    cplx is2 = cdiv(cmk(0.0, 0.5), s);  // i / (2 s)
    cplx sl = cmul(cmul(el, is2), w), dl = cmul(cscale(el, 0.5), w);
    cplx sr = cmul(cmul(er, is2), w), dr = cmul(cscale(er, -0.5), w);
    if (g.comps == 2 && !(i & 1)) {
      const cplx fl = wall_sigma_factor(g, i, s, km, true), fr = wall_sigma_factor(g, i, s, km, false);
      sl = cmul(sl, fl); dl = cmul(dl, fl);
      sr = cmul(sr, fr); dr = cmul(dr, fr);
    }
    if (combine) {
      W[(col_bl + m) * ldw + i] = cadd(sl, cmul(alpha, sr));
      W[(col_bl + M + m) * ldw + i] = cadd(dl, cmul(alpha, dr));
    } else {
      W[(col_bl + m) * ldw + i] = sl;
      W[(col_bl + M + m) * ldw + i] = dl;
      W[(col_br + m) * ldw + i] = sr;
      W[(col_br + M + m) * ldw + i] = dr;
    }
  }
}

// Fourier wall rows (2M x N, ld = ldc) for sources shifted by shift_x, wall at x0:
// f-row = D^ - i w S^, fn-row = T^ - i w D*^, times the source weights.
__global__ void k_fill_c(DevGeom g, const cplx* k, int M, double shift_x, double x0, cplx* C, int64_t ldc) {
  const int64_t tot = g.n * (int64_t)M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e % M);
    const int64_t j = e / M;
    const cplx km = k[m];
    const cplx s = sqrt_branch(g.omega, km);
    const double sx = g.x[j] + shift_x, sy = g.y[j], nx = g.nx[j], ny = g.ny[j];
    const double sg = sx - x0 > 0.0 ? 1.0 : -1.0;
    const double ax = fabs(sx - x0);
    // base = e^{-i k y} e^{i s |x - x0|} / (4 pi)
    cplx base = cmul(cexp(cmk(km.y * sy, -km.x * sy)), cexp(cmk(-s.y * ax, s.x * ax)));
    base = cscale(base, 1.0 / (4.0 * HBS_PI));
    cplx s_hat = cdiv(cmul(cmk(0.0, 1.0), base), s);
    cplx kos = cdiv(km, s);
    cplx d_hat = cmul(base, cadd(cmk(-sg * nx, 0.0), cscale(kos, ny)));
    cplx dstar_hat = cscale(base, sg);
    cplx t_hat = cmul(cmul(cmk(0.0, 1.0), base), csub(cscale(s, nx), cscale(km, sg * ny)));
    const cplx iw = cmk(0.0, g.omega);
    cplx f = csub(d_hat, cmul(iw, s_hat));
    cplx fn = csub(t_hat, cmul(iw, dstar_hat));
    if (g.comps == 2) {  // the pair: single-layer columns w [S^; D*^], double-layer [D^; T^]
      f = (j & 1) ? d_hat : cscale(s_hat, g.omega);
      fn = (j & 1) ? t_hat : cscale(dstar_hat, g.omega);
    }
    const double w = g.w[j];
    C[j * ldc + m] = cscale(f, w);
    C[j * ldc + M + m] = cscale(fn, w);
  }
}

// Bragg sampling rows for one image shift: rows (4S) = [u(x_s, +y0) | u(x_s, -y0) |
// u_y(x_s, +y0) | u_y(x_s, -y0)], columns = boundary nodes; entry = kernel * weight.
__global__ void k_fill_samples(DevGeom g, int S, double d, double y0, double shift_x, cplx* E, int64_t lde) {
  const int64_t tot = g.n * (int64_t)(4 * S);
  const double omega = g.omega;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % (4 * S));
    const int64_t j = e / (4 * S);
    const int s = r % S, kind = r / S;  // 0: u(+y0), 1: u(-y0), 2: u_y(+y0), 3: u_y(-y0)
    const double tx = -0.5 * d + (s + 0.5) * d / S;
    const double ty = (kind == 0 || kind == 2) ? y0 : -y0;
    const double sx = g.x[j] + shift_x, sy = g.y[j], nx = g.nx[j], ny = g.ny[j];
    cplx v;
    if (g.comps == 2) {
      v = pair_source_field(g, tx, ty, sx, sy, j, kind < 2 ? 0 : 2);
    } else if (kind < 2) {
      v = combined_kernel(tx, ty, sx, sy, nx, ny, omega, g.df);
    } else {
      // target y-derivative of dG/dn_y - i w G (see the oracle's derivation):
      // f' = -(i w/4) H1, f'' = -(i w^2/4)(H0 - H1/(w r)), g = f'/r, g' = (f'' - f'/r)/r
      double ddx = tx - sx, ddy = ty - sy;
      double r = sqrt(ddx * ddx + ddy * ddy);
      double z = omega * r;
      cplx h0, h1;
      hankel01(z, &h0, &h1, g.df);
      cplx f1 = cmul(cmk(0.0, -0.25 * omega), h1);
      cplx f2 = cmul(cmk(0.0, -0.25 * omega * omega), csub(h0, cscale(h1, 1.0 / z)));
      cplx gg = cscale(f1, 1.0 / r);
      cplx gp = cscale(csub(f2, cscale(f1, 1.0 / r)), 1.0 / r);
      double dn = ddx * nx + ddy * ny;
      cplx t1 = cscale(gp, -(ddy / r) * dn);
      cplx t2 = cscale(gg, -ny);
      cplx t3 = cmul(cmk(0.0, -omega * ddy), gg);
      v = cadd(cadd(t1, t2), t3);
    }
    E[j * lde + r] = cscale(v, g.w[j]);
  }
}

// Wall-potential contributions to the Bragg samples for one contour:
// SL, SR (4S x 2M), columns [mu (M) | nu (M)], same row layout as k_fill_samples.
__global__ void k_fill_wall_samples(const cplx* k, const cplx* wk, int M, int S, double d, double y0, double omega,
                                    cplx* SL, cplx* SR) {
  const int64_t tot = (int64_t)(4 * S) * M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % (4 * S));
    const int m = (int)(e / (4 * S));
    const int s = r % S, kind = r / S;
    const double tx = -0.5 * d + (s + 0.5) * d / S;
    const double ty = (kind == 0 || kind == 2) ? y0 : -y0;
    const cplx km = k[m], w = wk[m];
    const cplx sq = sqrt_branch(omega, km);
    cplx eky = cexp(cmk(-km.y * ty, km.x * ty));
    double al = tx + 0.5 * d, ar = 0.5 * d - tx;
    cplx el = cmul(eky, cexp(cmk(-sq.y * al, sq.x * al)));
    cplx er = cmul(eky, cexp(cmk(-sq.y * ar, sq.x * ar)));
    cplx is2 = cdiv(cmk(0.0, 0.5), sq);
    cplx sl = cmul(el, is2), dl = cscale(el, 0.5);
    cplx sr = cmul(er, is2), dr = cscale(er, -0.5);
    if (kind >= 2) {
      cplx ik = cmk(-km.y, km.x);
      sl = cmul(ik, sl); dl = cmul(ik, dl); sr = cmul(ik, sr); dr = cmul(ik, dr);
    }
    const int64_t ld = 4 * S;
    SL[(int64_t)m * ld + r] = cmul(sl, w);
    SL[(int64_t)(M + m) * ld + r] = cmul(dl, w);
    SR[(int64_t)m * ld + r] = cmul(sr, w);
    SR[(int64_t)(M + m) * ld + r] = cmul(dr, w);
  }
}

// Neighbour interaction matrix, transposed: Mt (m x N, ld = m).  Rows: image -1 near
// points (A_{-1}(i, near)), image +1 near points, then combined-layer (dG/dn - i w G)
// proxy sources on the neighbour circle (centre cx, cy; radius R; np points; weight wp).
__global__ void k_fill_nb(DevGeom g, const int64_t* near_m, int nm, const int64_t* near_p, int npn, double d, double cx,
                          double cy, double R, int np, double wp, cplx* Mt) {
  extern __shared__ double sdir[];  // 2 np doubles: proxy directions, once per block
  for (int p = threadIdx.x; p < np; p += blockDim.x) sincos(2.0 * HBS_PI * (double)p / (double)np, &sdir[np + p], &sdir[p]);
  __syncthreads();
  const int m = nm + npn + np;
  const int64_t tot = (int64_t)m * g.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % m);
    const int64_t i = e / m;
    cplx v;
    if (r < nm) {
      v = a_image_entry(g, i, near_m[r], -d);
    } else if (r < nm + npn) {
      v = a_image_entry(g, i, near_p[r - nm], d);
    } else {
      const int p = r - nm - npn;
      const double cs = sdir[p], sn = sdir[np + p];
      if (g.comps == 2) {
        v = cscale(proxy_row_entry(g, i, cx + R * cs, cy + R * sn, cs, sn, g.omega), wp);
      } else {
        cplx gg, dg;
        proxy_kernels(g.x[i], g.y[i], cx + R * cs, cy + R * sn, cs, sn, g.omega, &gg, &dg, g.df);
        v = cscale(cadd(dg, cmul(cmk(0.0, -g.omega), gg)), wp);
      }
    }
    Mt[i * (int64_t)m + r] = v;
  }
}

// Rows J of the image blocks: Rm = A_{-1}(J, :), Rp = A_{+1}(J, :) (l x N, ld = l).
__global__ void k_fill_r(DevGeom g, const int64_t* J, int l, double d, cplx* Rm, cplx* Rp) {
  const int64_t tot = (int64_t)l * g.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % l);
    const int64_t j = e / l;
    Rm[e] = a_image_entry(g, J[r], j, -d);
    Rp[e] = a_image_entry(g, J[r], j, d);
  }
}

// ---------------------------------------------------------------------------
// Multi-CTA column-pivoted QR for one large matrix (m x n, n large).  The host runs
// one step per pivot: k_bq_pivot (one block) picks the pivot, swaps it into place and
// forms the reflector; k_bq_update (grid over columns) applies it and downdates norms.
// State lives in BigQrState on the device.
// ---------------------------------------------------------------------------
__global__ void k_bq_norms(const cplx* A, int64_t m, int64_t n, double* nrm, double* nref, int* perm) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp; j < n; j += nwarps) {
    double s = 0.0;
    for (int64_t i = lane; i < m; i += 32) s += cabs2(A[j * m + i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) { nrm[j] = s; nref[j] = s; perm[j] = (int)j; }
  }
}

// partial argmax over columns [s, n): per-block result into partial arrays
__global__ void k_bq_argmax(const double* nrm, int64_t s, int64_t n, const BigQrState* st, double* pv, int* pi) {
  __shared__ double redv[32];
  __shared__ int redi[32];
  double best = -1.0;
  int bi = 0x7fffffff;
  if (!st->done) {
    for (int64_t j = s + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
      double v = nrm[j];
      if (v > best || (v == best && (int)j < bi)) { best = v; bi = (int)j; }
    }
  }
  double v;
  int i;
  block_argmax<256>(best, bi, redv, redi, &v, &i);
  if (threadIdx.x == 0) { pv[blockIdx.x] = v; pi[blockIdx.x] = i; }
}

__global__ void k_bq_pivot(cplx* A, int64_t m, int64_t s, double* nrm, double* nref, int* perm, const double* pv,
                           const int* pi, int nparts, BigQrState* st, double tol) {
  __shared__ double redv[32];
  __shared__ int redi[32];
  __shared__ double redsig[256];
  if (st->done) return;
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int q = threadIdx.x; q < nparts; q += blockDim.x) {
    if (pv[q] > best || (pv[q] == best && pi[q] < bi)) { best = pv[q]; bi = pi[q]; }
  }
  double v;
  int p;
  block_argmax<256>(best, bi, redv, redi, &v, &p);
  if (s == 0 && threadIdx.x == 0) st->r00 = sqrt(v);
  __syncthreads();
  const double r00 = st->r00;
  // |R_ss| <= tol |R_00|, compared squared (as the persistent QR does)
  if (!(r00 > 0.0) || !(v >= 0.0) || v <= (tol * r00) * (tol * r00) || s >= m) {
    if (threadIdx.x == 0) { st->done = 1; st->rank = (int)s; }
    return;
  }
  if (p != s) {
    cplx* cs = A + s * m;
    cplx* cp = A + (int64_t)p * m;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) { cplx t = cs[i]; cs[i] = cp[i]; cp[i] = t; }
    if (threadIdx.x == 0) {
      double t = nrm[s]; nrm[s] = nrm[p]; nrm[p] = t;
      t = nref[s]; nref[s] = nref[p]; nref[p] = t;
      int ti = perm[s]; perm[s] = perm[p]; perm[p] = ti;
    }
  }
  __syncthreads();
  cplx* cs = A + s * m;
  double sig = 0.0;
  for (int64_t i = s + 1 + threadIdx.x; i < m; i += blockDim.x) sig += cabs2(cs[i]);
  sig = block_sum_warp0<256>(sig, redsig);
  if (threadIdx.x == 0) {
    cplx v0, beta;
    double tau;
    householder_scalars(cs[s], sig, &v0, &beta, &tau);
    st->v0 = v0;
    st->tau = tau;
    cs[s] = beta;
    st->rank = (int)(s + 1);
  }
}

__global__ void k_bq_update(cplx* A, int64_t m, int64_t n, int64_t s, double* nrm, double* nref, const BigQrState* st) {
  if (st->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const cplx v0 = st->v0;
  const double tau = st->tau;
  const cplx* cs = A + s * m;
  for (int64_t j = s + 1 + warp; j < n; j += nwarps) {
    cplx* cj = A + j * m;
    cplx w = cmk(0.0, 0.0);
    for (int64_t i = s + 1 + lane; i < m; i += 32) w = cfma(cconj(cs[i]), cj[i], w);
    for (int o = 16; o > 0; o >>= 1) {
      w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
      w.y += __shfl_xor_sync(0xffffffffu, w.y, o);
    }
    w = cfma(cconj(v0), cj[s], w);
    w = cscale(w, tau);
    cplx top = cfms(v0, w, cj[s]);
    for (int64_t i = s + 1 + lane; i < m; i += 32) cj[i] = cfms(cs[i], w, cj[i]);
    double t = nrm[j] - cabs2(top);
    if (t <= 0.0078125 * nref[j]) {
      double q = 0.0;
      for (int64_t i = s + 1 + lane; i < m; i += 32) q += cabs2(cj[i]);
      for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      t = q;
      if (lane == 0) nref[j] = q;
    }
    if (lane == 0) { cj[s] = top; nrm[j] = t; }
  }
}

// T = R11^{-1} R12 for the big QR: one warp per column of R12.
__global__ void k_bq_tsolve(const cplx* A, int64_t m, int64_t n, int k, cplx* T) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < n - k; c += nwarps) {
    const cplx* r12 = A + (k + c) * m;
    cplx* tc = T + c * (int64_t)k;
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
}

int big_row_id(cplx* Mt, int64_t m, int64_t n, double tol, int* perm, cplx* T, int max_rank, cudaStream_t s) {
  const int kcap = (int)std::min<int64_t>(std::min<int64_t>(m, n), max_rank);
  std::vector<PqrSpec> sp{{Mt, m, n, kcap, perm, T}};
  PqrOut out;
  pqr_run(sp, tol, s, out);
  return out.rank[0];
}

}  // namespace hbs

namespace hbs {

// ---------------------------------------------------------------------------
// Compression of the periodizer blocks by interpolative decompositions computed on a
// subsample of the boundary points (their columns and rows are smooth functions of the
// boundary point, so the decomposition found on a fine subsample holds on all N points;
// a second, disjoint subsample checks it).
// ---------------------------------------------------------------------------

// out[i + c ldo] = src[sub[i] + c lds]: rows `sub` of src (all ncol columns).
__global__ void k_gather_subrows(const cplx* src, int64_t lds, const int64_t* sub, int ns, int ncol, cplx* out,
                                 int64_t ldo) {
  const int64_t tot = (int64_t)ns * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % ns);
    const int64_t c = e / ns;
    out[i + c * ldo] = src[sub[i] + c * lds];
  }
}

// out[i + (col0 + r) ldo] = src[r + sub[i] lds] for r < nrows: columns `sub` of src, transposed.
__global__ void k_gather_subcols_t(const cplx* src, int64_t lds, int nrows, const int64_t* sub, int ns, cplx* out,
                                   int64_t ldo, int col0) {
  const int64_t tot = (int64_t)ns * nrows;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % ns);
    const int r = (int)(e / ns);
    out[i + (int64_t)(col0 + r) * ldo] = src[r + sub[i] * lds];
  }
}

// out[t + j ldo] = refs[t].base[j refs[t].ld]: selected rows of several matrices, stacked.
__global__ void k_gather_rowrefs(const RowRef* refs, int nsel, int64_t ncol, cplx* out, int64_t ldo) {
  const int64_t tot = (int64_t)nsel * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e % nsel);
    const int64_t j = e / nsel;
    out[t + j * ldo] = refs[t].base[j * refs[t].ld];
  }
}

// Row expansion by recipe: out[o, c] = in[idx, c] (kind 0), or
// sum_i T1[i, idx] in[off1 + i, c] (kind 1), or sum_i T2[i, idx] in[off2 + i, c] (kind 2).
__global__ void k_expand_rows(const cplx* in, int64_t ldi, int ncol, const int2* recipe, int nout, const cplx* T1,
                              int r1, int off1, const cplx* T2, int r2, int off2, cplx* out, int64_t ldo) {
  const int64_t tot = (int64_t)nout * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int o = (int)(e % nout);
    const int64_t c = e / nout;
    const int2 rc = recipe[o];
    const cplx* col = in + c * ldi;
    cplx v;
    if (rc.x == 0) {
      v = col[rc.y];
    } else {
      const cplx* T = rc.x == 1 ? T1 : T2;
      const int r = rc.x == 1 ? r1 : r2, off = rc.x == 1 ? off1 : off2;
      const cplx* tc = T + (int64_t)rc.y * r;
      v = cmk(0, 0);
      for (int i = 0; i < r; ++i) v = cfma(tc[i], col[off + i], v);
    }
    out[o + c * ldo] = v;
  }
}

// Column expansion by recipe: out[:, o] = in[:, idx] (kind 0), or sum_i T[i, idx] in[:, col(i)]
// with col(i) = skel ? skel[i] : off + i (kind 1).
__global__ void k_expand_cols(const cplx* in, int64_t ldi, int nrow, const int2* recipe, int nout, const cplx* T, int r,
                              int off, const int* skel, cplx* out, int64_t ldo) {
  const int64_t tot = (int64_t)nrow * nout;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int rw = (int)(e % nrow);
    const int o = (int)(e / nrow);
    const int2 rc = recipe[o];
    cplx v;
    if (rc.x == 0) {
      v = in[rw + (int64_t)rc.y * ldi];
    } else {
      const cplx* tc = T + (int64_t)rc.y * r;
      v = cmk(0, 0);
      for (int i = 0; i < r; ++i) {
        const int cc = skel ? skel[i] : off + i;
        v = cfma(tc[i], in[rw + (int64_t)cc * ldi], v);
      }
    }
    out[rw + (int64_t)o * ldo] = v;
  }
}

// acc[0] += |a - b|^2, acc[1] += |b|^2 over an nrow x ncol block.
__global__ void k_diff_norm2(const cplx* a, int64_t lda, const cplx* b, int64_t ldb, int nrow, int ncol, double* acc) {
  __shared__ double red[2][32];
  double s0 = 0.0, s1 = 0.0;
  const int64_t tot = (int64_t)nrow * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int rw = (int)(e % nrow);
    const int64_t c = e / nrow;
    const cplx x = a[rw + c * lda], y = b[rw + c * ldb];
    s0 += cabs2(csub(x, y));
    s1 += cabs2(y);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = s0; red[1][threadIdx.x >> 5] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t0 += red[0][w]; t1 += red[1][w]; }
    atomicAdd(&acc[0], t0);
    atomicAdd(&acc[1], t1);
  }
}

}  // namespace hbs

namespace hbs {

// Column-pivoted QR / ID of several large matrices (the top tree levels) in one
// persistent launch (pqr.cu).
std::vector<int> big_row_id_batched(std::vector<BigQrJobSpec>& specs, double tol, cudaStream_t s) {
  std::vector<PqrSpec> sp;
  for (auto& j : specs) sp.push_back({j.A, j.m, j.n, (int)std::min(j.m, j.n), j.perm, j.T});
  PqrOut out;
  pqr_run(sp, tol, s, out);
  return out.rank;
}

}  // namespace hbs

namespace hbs {

// ---------------------------------------------------------------------------
// Entry-wise periodizer fills on index lists, so that the precomputed path only
// evaluates the subsample used by the interpolative decompositions and the skeleton
// rows / columns it keeps.
// ---------------------------------------------------------------------------

__global__ void k_contour_s(const cplx* k, int M, double omega, cplx* s, cplx* si) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
    const cplx v = sqrt_branch(omega, k[m]);
    s[m] = v;
    si[m] = cdiv(cmk(1.0, 0.0), v);
  }
}

// Column `col` of Y = [B_L^0 | B_R^0 | B_L^1 | B_R^1] at boundary node i (each block [mu | nu]):
// e^{i k_m y} e^{i s a} as one exponential, with s and 1/s from the per-node tables.
__device__ __forceinline__ cplx b_entry(const DevGeom& g, const ContourPtrs& cp, int M, double d, int64_t i, int col) {
  const int c = col / (4 * M), rem = col % (4 * M);
  const int side = rem / (2 * M), kind = (rem % (2 * M)) / M, m = rem % M;
  const cplx km = cp.k[c][m], w = cp.wk[c][m];
  const cplx s = cp.s[c][m];
  const double xi = g.x[i], yi = g.y[i];
  const double a = side == 0 ? xi + 0.5 * d : 0.5 * d - xi;
  cplx e = cexp(cmk(-km.y * yi - s.y * a, km.x * yi + s.x * a));
  if (g.comps == 2 && !(i & 1)) e = cmul(e, wall_sigma_factor(g, i, s, km, side == 0));
  if (kind == 0) {
    const cplx si = cp.si[c][m];  // (i / 2) / s
    return cmul(cmul(e, cmk(-0.5 * si.y, 0.5 * si.x)), w);
  }
  return cmul(cscale(e, side == 0 ? 0.5 : -0.5), w);
}

// Row `a` of C = [C_L^0; C_R^0; C_L^1; C_R^1] (each block [f; fn] rows) at boundary node j.
__device__ __forceinline__ cplx c_entry(const DevGeom& g, const ContourPtrs& cp, int M, double d, int a, int64_t j) {
  const int c = a / (4 * M), rem = a % (4 * M);
  const int side = rem / (2 * M), kind = (rem % (2 * M)) / M, m = rem % M;
  const double shift_x = side == 0 ? d : -d, x0 = side == 0 ? -0.5 * d : 0.5 * d;
  const cplx km = cp.k[c][m];
  const cplx s = cp.s[c][m], si = cp.si[c][m];
  const double sx = g.x[j] + shift_x, sy = g.y[j], nx = g.nx[j], ny = g.ny[j];
  const double sg = sx - x0 > 0.0 ? 1.0 : -1.0;
  const double ax = fabs(sx - x0);
  cplx base = cexp(cmk(km.y * sy - s.y * ax, -km.x * sy + s.x * ax));  // e^{-i k_m y} e^{i s |x - x0|}
  base = cscale(base, g.w[j] / (4.0 * HBS_PI));
  const cplx iw = cmk(0.0, g.omega);
  // transmission: w S^, w D*^ (single layer) or D^, T^ (double layer)
  const bool pair = g.comps == 2, tau = (j & 1) != 0;
  if (kind == 0) {
    cplx s_hat = cmul(cmul(cmk(0.0, 1.0), base), si);
    cplx d_hat = cmul(base, cadd(cmk(-sg * nx, 0.0), cscale(cmul(km, si), ny)));
    if (pair) return tau ? d_hat : cscale(s_hat, g.omega);
    return csub(d_hat, cmul(iw, s_hat));
  }
  cplx dstar_hat = cscale(base, sg);
  cplx t_hat = cmul(cmul(cmk(0.0, 1.0), base), csub(cscale(s, nx), cscale(km, sg * ny)));
  if (pair) return tau ? t_hat : cscale(dstar_hat, g.omega);
  return csub(t_hat, cmul(iw, dstar_hat));
}

// Row `r` of the Bragg sampling rows E (3 images x [u(+y0) | u(-y0) | u_y(+y0) | u_y(-y0)]).
__device__ __forceinline__ cplx e_entry(const DevGeom& g, int S, double d, double y0, int r, int64_t j) {
  const int jj = r / (4 * S), rr = r % (4 * S);
  const int s = rr % S, kind = rr / S;
  const double tx = -0.5 * d + (s + 0.5) * d / S;
  const double ty = (kind == 0 || kind == 2) ? y0 : -y0;
  const double sx = g.x[j] + (jj - 1) * d, sy = g.y[j], nx = g.nx[j], ny = g.ny[j];
  const double omega = g.omega;
  cplx v;
  if (g.comps == 2) {
    v = pair_source_field(g, tx, ty, sx, sy, j, kind < 2 ? 0 : 2);
  } else if (kind < 2) {
    v = combined_kernel(tx, ty, sx, sy, nx, ny, omega, g.df);
  } else {
    double ddx = tx - sx, ddy = ty - sy;
    double rr2 = sqrt(ddx * ddx + ddy * ddy);
    double z = omega * rr2;
    cplx h0, h1;
    hankel01(z, &h0, &h1, g.df);
    cplx f1 = cmul(cmk(0.0, -0.25 * omega), h1);
    cplx f2 = cmul(cmk(0.0, -0.25 * omega * omega), csub(h0, cscale(h1, 1.0 / z)));
    cplx gg = cscale(f1, 1.0 / rr2);
    cplx gp = cscale(csub(f2, cscale(f1, 1.0 / rr2)), 1.0 / rr2);
    double dn = ddx * nx + ddy * ny;
    v = cadd(cadd(cscale(gp, -(ddy / rr2) * dn), cscale(gg, -ny)), cmul(cmk(0.0, -omega * ddy), gg));
  }
  return cscale(v, g.w[j]);
}

// out[i + c ld] = entry at (pts[i], c) for kinds 0 (B columns), 1 (C rows), 2 (E rows),
// all `nfam` members of the family; used for the subsampled decompositions.
__global__ void k_fill_family_sub(DevGeom g, ContourPtrs cp, int M, double d, int S, double y0, int family,
                                  const int64_t* pts, int np, int nfam, cplx* out, int64_t ld) {
  const int64_t tot = (int64_t)np * nfam;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % np), c = (int)(e / np);
    const int64_t p = pts[i];
    cplx v = family == 0 ? b_entry(g, cp, M, d, p, c) : (family == 1 ? c_entry(g, cp, M, d, c, p)
                                                                    : e_entry(g, S, d, y0, c, p));
    out[i + (int64_t)c * ld] = v;
  }
}

// Selected members over all N nodes.  B columns: out[i + t ld] (N x nsel);
// C / E rows: out[t + i ld] (nsel x N, e.g. rows of Rsel).
__global__ void k_fill_family_sel(DevGeom g, ContourPtrs cp, int M, double d, int S, double y0, int family,
                                  const int* sel, int nsel, cplx* out, int64_t ld) {
  const int64_t tot = g.n * (int64_t)nsel;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    if (family == 0) {
      const int64_t i = e % g.n;
      const int t = (int)(e / g.n);
      out[i + (int64_t)t * ld] = b_entry(g, cp, M, d, i, sel[t]);
    } else {
      const int t = (int)(e % nsel);
      const int64_t i = e / nsel;
      out[t + i * ld] = family == 1 ? c_entry(g, cp, M, d, sel[t], i) : e_entry(g, S, d, y0, sel[t], i);
    }
  }
}

}  // namespace hbs

namespace hbs {

// out (cols x rows, column-major) = in^T for in (rows x cols, column-major).
__global__ void k_transpose(const cplx* in, int64_t rows, int64_t cols, cplx* out) {
  const int64_t tot = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e % cols, r = e / cols;
    out[c + r * cols] = in[r + c * rows];
  }
}

}  // namespace hbs

namespace hbs {

// out[i + k N] = exp(i w ((x_i - cx) cos phi_k + (y_i - cy) sin phi_k)), phi_k = 2 pi k / K.
__global__ void k_fill_dirs(DevGeom g, double cx, double cy, int K, cplx* out) {
  const int64_t tot = g.n * (int64_t)K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % g.n;
    const int k = (int)(e / g.n);
    double sn, cs;
    sincospi(2.0 * (double)k / (double)K, &sn, &cs);
    cplx v = cexp_i(g.omega * ((g.x[i] - cx) * cs + (g.y[i] - cy) * sn));
    if (g.comps == 2 && !(i & 1)) {  // transmission sigma row: -(d/dn) / w = -i (n . dir)
      const double f = -(g.nx[i] * cs + g.ny[i] * sn);
      v = cmk(-f * v.y, f * v.x);
    }
    out[e] = v;
  }
}

}  // namespace hbs
