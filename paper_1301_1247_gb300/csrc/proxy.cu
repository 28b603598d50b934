// Second periodizer: proxy points and wall discrepancies (hbs_solve_proxy).
//
// The paper periodizes with Sommerfeld-contour wall potentials (Secs. 2.2-2.4); this solve
// periodizes the same discrete obstacle another way, so that the two schemes' Bragg
// amplitudes check each other.  It keeps the handle's compressed A^{-1} (Sec. 4) and the
// neighbour factors A_{+-1} ~ P R_{+-1} (Sec. 3.2, Def. 3.1).  The unit cell is cut to the box
// |x| <= d/2, |y| <= h, h = max|y| + d/8, and inside it
//     u = sum_{|j| <= 1} alpha^j (D - i w S)_{dOmega + j d} eta + sum_p c_p phi_p,
// phi_p the combined-field source at proxy point p of a circle of radius
// R_p = max(0.75 d, 1.4 * half-diagonal of the box).  Unknowns besides eta: the proxy
// strengths c and the outgoing Rayleigh-Bloch coefficients a_n (above y = h) and b_n (below
// y = -h), |n| <= K = ceil(w d / pi) + 40.  Equations: u = -u_inc on dOmega; at M_w = 40
// Gauss-Legendre heights on the walls, u(-d/2) - u(d/2)/alpha = 0 and the same for u_x
// (the images telescope to alpha Phi_1(L) - alpha^{-2} Phi_{-1}(R)); at M_t = 2(2K+1) + 8
// points of each line y = +-h, u and u_y equal those of the expansions.
//
// With eta = A^{-1}(f - L zeta - Phi c) (L = [alpha^{-1} P | alpha P], zeta = R eta as in the
// Woodbury form of Sec. 3.2), each Bloch phase leaves a small rectangular system in
// (zeta, c, a, b), solved in the least-squares sense.  Per call:
//   1. the row operators (R_{-1}, R_1, the wall rows of the images +-1, the line rows of the
//      images -1, 0, 1) as one (2l + 4 M_w + 12 M_t) x N matrix, and the proxy columns;
//   2. X = A^{-1} [P | Phi | f(theta)] in one apply of the compressed inverse;
//   3. Y = Rows X in one GEMM;
//   4. per Bloch phase, the system assembled from Y (k_px_assemble) and solved by Householder
//      QR (k_px_lsq, one CTA per phase; column-equilibrated);
//   5. c_n, d_n of the propagating orders referred to y = +-y0, and the flux balance.
// Every step is FP64.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>

#include "dense_kernels.cuh"
#include "profile.hpp"
#include "qp_kernels.cuh"

namespace hbs {

namespace {

constexpr int kWallNodes = 40;
constexpr int kLsqNT = 512;

struct PxRow {
  double tx, ty;
  double shift;  // x-shift of the sources (image j d)
  int kind;      // 0: u, 1: u_x, 2: u_y
};

// dG/dn_s - i w G at target t from a source s with normal n, or its target x- or y-derivative.
// With f(r) = (i/4) H0(w r): f' = -(i w/4) H1, f'' = -(i w^2/4)(H0 - H1/(w r)), g = f'/r,
// g' = (f'' - f'/r)/r and e = t - s:  d/dt_i [dG/dn_s] = -g' (e_i/r)(e.n) - g n_i,
// d/dt_i [G] = g e_i.
__device__ cplx px_kernel(double tx, double ty, double sx, double sy, double nx, double ny, double omega, int kind) {
  const double ex = tx - sx, ey = ty - sy;
  const double r = sqrt(ex * ex + ey * ey);
  const double z = omega * r;
  cplx h0, h1;
  hankel01(z, &h0, &h1, false);
  const double en = ex * nx + ey * ny;
  if (kind == 0) {
    const cplx dgdn = cscale(cmul(cmk(0.0, 0.25 * omega), h1), en / r);
    const cplx g = cmul(cmk(0.0, 0.25), h0);
    return csub(dgdn, cmul(cmk(0.0, omega), g));
  }
  const cplx f1 = cmul(cmk(0.0, -0.25 * omega), h1);
  const cplx f2 = cmul(cmk(0.0, -0.25 * omega * omega), csub(h0, cscale(h1, 1.0 / z)));
  const cplx g = cscale(f1, 1.0 / r);
  const cplx gp = cscale(csub(f2, cscale(f1, 1.0 / r)), 1.0 / r);
  const double ei = kind == 1 ? ex : ey, ni = kind == 1 ? nx : ny;
  cplx v = cscale(gp, -(ei / r) * en);
  v = csub(v, cscale(g, ni));
  return csub(v, cmul(cmk(0.0, omega * ei), g));
}

// Rows r0 .. r0 + nr of the row operator: the field of the boundary layer (shifted by the
// row's image) at the row's target, times the trapezoid weight of the source node.
__global__ void k_px_rows(DevGeom g, const PxRow* rows, int nr, int r0, cplx* R, int64_t ldr) {
  const int64_t tot = (int64_t)nr * g.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % nr);
    const int64_t j = e / nr;
    const PxRow q = rows[r];
    // the combined layer (sound-soft), or the layer of unknown j's density (transmission)
    const cplx k = g.comps == 2 ? pair_source_field(g, q.tx, q.ty, g.x[j] + q.shift, g.y[j], j, q.kind)
                                : px_kernel(q.tx, q.ty, g.x[j] + q.shift, g.y[j], g.nx[j], g.ny[j], g.omega, q.kind);
    R[(int64_t)(r0 + r) + j * ldr] = cscale(k, g.w[j]);
  }
}

// out(r, p) = phi_p at row r's target (value or derivative), rows x mp, ld = nr.
__global__ void k_px_proxy_rows(const PxRow* rows, int nr, const double* p4, int mp, double omega, cplx* out) {
  const int64_t tot = (int64_t)nr * mp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % nr), p = (int)(e / nr);
    const PxRow q = rows[r];
    out[e] = px_kernel(q.tx, q.ty, p4[4 * p], p4[4 * p + 1], p4[4 * p + 2], p4[4 * p + 3], omega, q.kind);
  }
}

// Right-hand sides X(:, 0:l) = P, X(:, l:l+mp) = phi_p at the nodes, X(:, l+mp+q) = -u_inc(theta_q)
// (transmission: the row functionals of phi_p and of -u_inc, Sec. 5).
__global__ void k_px_rhs(DevGeom g, const cplx* P, int l, const double* p4, int mp, const double* kx,
                         const double* ky, int nq, cplx* X) {
  const int64_t n = g.n;
  const int64_t tot = n * (int64_t)(l + mp + nq);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n;
    const int c = (int)(e / n);
    cplx v;
    if (c < l) {
      v = P[e];
    } else if (c < l + mp) {
      const int p = c - l;
      v = g.comps == 2 ? proxy_row_entry(g, i, p4[4 * p], p4[4 * p + 1], p4[4 * p + 2], p4[4 * p + 3], g.omega)
                       : px_kernel(g.x[i], g.y[i], p4[4 * p], p4[4 * p + 1], p4[4 * p + 2], p4[4 * p + 3], g.omega, 0);
    } else {
      const int q = c - l - mp;
      const cplx u = cexp_i(kx[q] * g.x[i] + ky[q] * g.y[i]);
      v = cmk(-u.x, -u.y);
      if (g.comps == 2 && !(i & 1)) {  // sigma row: +(du/dn) / w = i (kx n_x + ky n_y) u / w
        const double f = (kx[q] * g.nx[i] + ky[q] * g.ny[i]) / g.omega;
        v = cmk(-f * u.y, f * u.x);
      }
    }
    X[e] = v;
  }
}

struct PxDims {
  int l, mp, mw, mt, nu, kk;   // neighbour rank, proxies, wall nodes, line points, 2K+1, K
  int rtot, ycols;             // rows of Y, columns of Y (l + mp + Q)
  int ms, ns;                  // Schur system: rows, columns
  double d, h, omega;
  int off_wl, off_wr, off_t;   // row offsets in Y of the wall (+1 at L, -1 at R) and line blocks
};

struct PxGroup {
  cplx alpha;
  double kap0;   // kappa_0 of the group's first angle
  int q;         // angles
  int col0;      // their first column among the f columns of X / Y
  int64_t s_off, r_off;  // this group's system (ms x ns) and right-hand sides (ms x q)
};

// S (ms x ns) and R (ms x q) of one Bloch phase (blockIdx.y) from Y, the proxy blocks at the
// walls (QL, QR: 2 mw x mp) and on the lines (VP: 4 mt x mp), and the Rayleigh-Bloch columns.
// Unknowns [zeta_- (l) | zeta_+ (l) | c (mp) | a (nu) | b (nu)], rows [R rows (2l) | wall
// rows (2 mw) | line rows (4 mt)].
__global__ void k_px_assemble(PxDims D, const PxGroup* groups, const cplx* Y, const cplx* QL, const cplx* QR,
                              const cplx* VP, const double* xline, cplx* S, cplx* R) {
  const PxGroup G = groups[blockIdx.y];
  const cplx a = G.alpha, ai = cdiv(cmk(1.0, 0.0), a);
  const cplx a2i = cmul(ai, ai);
  const int ms = D.ms, ns = D.ns, l = D.l, mp = D.mp;
  const int64_t ld = D.rtot;
  const int ncol = ns + G.q;
  const int64_t tot = (int64_t)ms * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % ms), c = (int)(e / ms);
    // the Y column this entry reads (zeta: P columns; c: proxy columns; rhs: f columns)
    int yc = -1;
    cplx zs = cmk(0.0, 0.0);  // alpha factor of L's block for zeta columns
    if (c < 2 * l) { yc = c % l; zs = c < l ? ai : a; }
    else if (c < 2 * l + mp) yc = l + (c - 2 * l);
    else if (c >= ns) yc = l + mp + G.col0 + (c - ns);
    // the combination of Y rows for this row: M Y(:, yc)
    cplx my = cmk(0.0, 0.0);
    cplx sub = cmk(0.0, 0.0);  // proxy block subtracted from the proxy columns
    if (r < 2 * l) {
      if (yc >= 0) my = Y[r + yc * ld];
    } else if (r < 2 * l + 2 * D.mw) {
      const int k = r - 2 * l;
      if (yc >= 0) my = csub(cmul(a, Y[D.off_wl + k + yc * ld]), cmul(a2i, Y[D.off_wr + k + yc * ld]));
      if (c >= 2 * l && c < 2 * l + mp) {
        const int p = c - 2 * l;
        sub = csub(QL[k + (int64_t)p * 2 * D.mw], cmul(ai, QR[k + (int64_t)p * 2 * D.mw]));
      }
    } else {
      const int k = r - 2 * l - 2 * D.mw;
      if (yc >= 0) {
        const cplx t0 = Y[D.off_t + k + yc * ld];
        const cplx t1 = Y[D.off_t + 4 * D.mt + k + yc * ld];
        const cplx t2 = Y[D.off_t + 8 * D.mt + k + yc * ld];
        my = cadd(cadd(cmul(ai, t0), t1), cmul(a, t2));
      }
      if (c >= 2 * l && c < 2 * l + mp) sub = VP[k + (int64_t)(c - 2 * l) * 4 * D.mt];
    }
    cplx v;
    if (c < 2 * l) {
      v = cmul(zs, my);
      if (r == c) v = cadd(v, cmk(1.0, 0.0));  // the -I of zeta = R eta, moved across
    } else if (c < 2 * l + mp) {
      v = csub(my, sub);
    } else if (c < ns) {
      // Rayleigh-Bloch columns: only the line rows
      v = cmk(0.0, 0.0);
      if (r >= 2 * l + 2 * D.mw) {
        const int k = r - 2 * l - 2 * D.mw;
        const int kind = k / D.mt;  // 0: top u, 1: top u_y, 2: bottom u, 3: bottom u_y
        const double x = xline[k % D.mt];
        const int cc = c - 2 * l - mp;
        const bool top = cc < D.nu;
        const int n = (top ? cc : cc - D.nu) - D.kk;
        if (top == (kind < 2)) {
          const double kap = G.kap0 + 2.0 * M_PI * n / D.d;
          const double v2 = D.omega * D.omega - kap * kap;
          const cplx kn = fabs(v2) <= 1e-12 * D.omega * D.omega ? cmk(0.0, 0.0)
                          : (v2 >= 0.0 ? cmk(sqrt(v2), 0.0) : cmk(0.0, sqrt(-v2)));
          const cplx ex = cexp_i(kap * x);
          if (kind == 0 || kind == 2) v = ex;
          else v = cmul(cmul(cmk(0.0, kind == 1 ? 1.0 : -1.0), kn), ex);
        }
      }
    } else {
      v = my;
    }
    if (c < ns) S[G.s_off + r + (int64_t)c * ms] = v;
    else R[G.r_off + r + (int64_t)(c - ns) * ms] = v;
  }
}

// Least squares min ||S z - R|| by Householder QR, one CTA per Bloch phase: columns
// equilibrated first (their scales undone at the end), then for each column the reflector
// (kept in place below the diagonal) is applied to the remaining columns and to the right-hand
// sides, and R11 z = (Q^H R)(0:ns) is solved by back substitution.  z overwrites R(0:ns, :).
__global__ void __launch_bounds__(kLsqNT) k_px_lsq(PxDims D, const PxGroup* groups, cplx* S, cplx* R, double* colsc) {
  __shared__ double red[kLsqNT];
  __shared__ cplx s_beta, s_inv;
  __shared__ double s_tau;
  const PxGroup G = groups[blockIdx.x];
  const int ms = D.ms, ns = D.ns, q = G.q;
  cplx* A = S + G.s_off;
  cplx* B = R + G.r_off;
  double* sc = colsc + (int64_t)blockIdx.x * ns;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kLsqNT / 32;
  // column equilibration
  for (int c = warp; c < ns; c += NW) {
    double s2 = 0.0;
    for (int i = lane; i < ms; i += 32) s2 += cabs2(A[i + (int64_t)c * ms]);
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    const double f = s2 > 0.0 ? 1.0 / sqrt(s2) : 1.0;
    for (int i = lane; i < ms; i += 32) A[i + (int64_t)c * ms] = cscale(A[i + (int64_t)c * ms], f);
    if (lane == 0) sc[c] = f;
  }
  __syncthreads();
  for (int k = 0; k < ns; ++k) {
    cplx* ak = A + (int64_t)k * ms;
    double s2 = 0.0;
    for (int i = k + 1 + tid; i < ms; i += kLsqNT) s2 += cabs2(ak[i]);
    s2 = block_sum<kLsqNT>(s2, red);
    if (tid == 0) {
      const cplx x0 = ak[k];
      const double nrm = sqrt(cabs2(x0) + s2);
      if (nrm == 0.0) {
        s_tau = 0.0;
        s_beta = cmk(0.0, 0.0);
      } else {
        // v = [1; x(k+1:)/(x0 - beta)], beta = -e^{i arg x0} ||x||, tau = (beta - x0)/beta
        const double ax0 = sqrt(cabs2(x0));
        const cplx ph = ax0 > 0.0 ? cscale(x0, 1.0 / ax0) : cmk(1.0, 0.0);
        const cplx beta = cscale(ph, -nrm);
        const cplx den = csub(x0, beta);
        s_beta = beta;
        s_tau = 1.0 + ax0 / nrm;  // real for this choice of beta
        s_inv = cdiv(cmk(1.0, 0.0), den);  // scales the tail so that v(k) = 1
      }
    }
    __syncthreads();
    const cplx inv = s_inv;
    const double tau = s_tau;
    if (tau != 0.0)
      for (int i = k + 1 + tid; i < ms; i += kLsqNT) ak[i] = cmul(ak[i], inv);
    if (tid == 0) ak[k] = s_beta;
    __syncthreads();
    // apply H = I - tau v v^H to the other columns and the right-hand sides
    if (tau != 0.0) {
      for (int c = k + 1 + warp; c < ns + q; c += NW) {
        cplx* y = c < ns ? A + (int64_t)c * ms : B + (int64_t)(c - ns) * ms;
        cplx w = lane == 0 ? y[k] : cmk(0.0, 0.0);
        for (int i = k + 1 + lane; i < ms; i += 32) w = cfma(cconj(ak[i]), y[i], w);
        for (int o = 16; o > 0; o >>= 1) {
          w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
          w.y += __shfl_xor_sync(0xffffffffu, w.y, o);
        }
        w = cscale(w, tau);
        if (lane == 0) y[k] = csub(y[k], w);
        for (int i = k + 1 + lane; i < ms; i += 32) y[i] = cfms(ak[i], w, y[i]);
      }
    }
    __syncthreads();
  }
  // back substitution, one warp per right-hand side
  for (int j = warp; j < q; j += NW) {
    cplx* b = B + (int64_t)j * ms;
    for (int i = ns - 1; i >= 0; --i) {
      cplx acc = cmk(0.0, 0.0);
      for (int t = i + 1 + lane; t < ns; t += 32) acc = cfma(A[i + (int64_t)t * ms], b[t], acc);
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) b[i] = cdiv(csub(b[i], acc), A[i + (int64_t)i * ms]);
      __syncwarp();
    }
    for (int i = lane; i < ns; i += 32) b[i] = cscale(b[i], sc[i]);
  }
}

struct PxAngle {
  int64_t z_off;    // this angle's solution in the right-hand-side pool
  int m;            // its order n is the group's mode n + m
  int n_min, n_max;
  int out_off;      // its first order in the output arrays
  double kap, k0;   // kappa_0 and omega |sin theta|
};

// c_n, d_n of the propagating orders referred to y = +-y0 (a_n, b_n times e^{i k_n (y0 - h)})
// and the flux error sum (k_n/k0)(|c_n|^2 + |d_n + delta_n0 e^{i k0 y0}|^2) - 1, one CTA per angle.
__global__ void k_px_bragg(PxDims D, const PxAngle* angles, const cplx* Z, double y0, cplx* cout, cplx* dout,
                           double* flux) {
  __shared__ double red[256];
  const PxAngle A = angles[blockIdx.x];
  const cplx* z = Z + A.z_off;
  double f = 0.0;
  for (int n = A.n_min + (int)threadIdx.x; n <= A.n_max; n += blockDim.x) {
    const int mode = n + A.m + D.kk;
    const double kap = A.kap + 2.0 * M_PI * n / D.d;
    double v2 = D.omega * D.omega - kap * kap;
    if (fabs(v2) <= 1e-12 * D.omega * D.omega) v2 = 0.0;
    const double kn = sqrt(fmax(v2, 0.0));
    const cplx ph = cexp_i(kn * (y0 - D.h));
    cplx an = cmk(0.0, 0.0), bn = cmk(0.0, 0.0);
    if (mode >= 0 && mode < D.nu) {
      an = cmul(z[2 * D.l + D.mp + mode], ph);
      bn = cmul(z[2 * D.l + D.mp + D.nu + mode], ph);
    }
    cout[A.out_off + n - A.n_min] = an;
    dout[A.out_off + n - A.n_min] = bn;
    const cplx bi = n == 0 ? cadd(bn, cexp_i(A.k0 * y0)) : bn;
    f += (kn / A.k0) * (cabs2(an) + cabs2(bi));
  }
  f = block_sum<256>(f, red);
  if (threadIdx.x == 0) flux[blockIdx.x] = fabs(f - 1.0);
}

// Gauss-Legendre nodes on [-1, 1] (Newton on the Legendre polynomial from the Chebyshev
// guesses cos(pi (i + 3/4) / (n + 1/2))).
std::vector<double> gauss_legendre(int n) {
  std::vector<double> x(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  std::sort(x.begin(), x.end());
  return x;
}

}  // namespace

void solve_angles_proxy(Handle& h, const double* theta, int64_t n_theta, Result& out, cudaStream_t s) {
  out.angles.assign(n_theta, AngleResult{});
  if (n_theta == 0) return;
  const int64_t N = h.N;
  const double d = h.d, omega = h.omega;
  const int l = h.nb_rank;
  double ymax = 0.0;
  for (double v : h.hy) ymax = std::max(ymax, std::fabs(v));
  PxDims D{};
  D.d = d;
  D.omega = omega;
  D.h = ymax + d / 8.0;
  const double rp = std::max(0.75 * d, 1.4 * std::hypot(0.5 * d, D.h));
  D.l = l;
  D.mp = std::max(100, 2 * (int)std::ceil(omega * rp) + 60);
  D.mw = kWallNodes;
  D.kk = (int)std::ceil(omega * d / M_PI) + 40;
  D.nu = 2 * D.kk + 1;
  D.mt = 2 * D.nu + 8;
  D.off_wl = 2 * l;
  D.off_wr = 2 * l + 2 * D.mw;
  D.off_t = 2 * l + 4 * D.mw;
  D.rtot = 2 * l + 4 * D.mw + 12 * D.mt;
  D.ms = 2 * l + 2 * D.mw + 4 * D.mt;
  D.ns = 2 * l + D.mp + 2 * D.nu;

  // group the angles by Bloch phase (as the Fourier-wall solve does)
  std::map<long long, std::vector<int64_t>> bykey;
  const double step = 2.0 * M_PI / d;
  for (int64_t i = 0; i < n_theta; ++i) {
    double kap = omega * std::cos(theta[i]);
    double r = std::fmod(kap, step);
    if (r < 0) r += step;
    bykey[std::llround(r / step * 1e9) % 1000000000LL].push_back(i);
  }
  std::vector<std::vector<int64_t>> groups;
  for (auto& kv : bykey) groups.push_back(kv.second);
  const int ng = (int)groups.size();
  const int nq = (int)n_theta;

  // rows: wall heights, line points, and their descriptors
  const std::vector<double> gl = gauss_legendre(D.mw);
  std::vector<double> xline(D.mt);
  for (int k = 0; k < D.mt; ++k) xline[k] = -0.5 * d + (k + 0.5) * d / D.mt;
  std::vector<PxRow> rows;  // rows of the boundary-layer operator after R_{-1}, R_1
  for (int side = 0; side < 2; ++side)      // image +1 at L, image -1 at R
    for (int kind = 0; kind < 2; ++kind)      // u, u_x
      for (int k = 0; k < D.mw; ++k)
        rows.push_back({side == 0 ? -0.5 * d : 0.5 * d, D.h * gl[k], side == 0 ? d : -d, kind});
  for (int j = -1; j <= 1; ++j)
    for (int kind = 0; kind < 4; ++kind)      // top u, top u_y, bottom u, bottom u_y
      for (int k = 0; k < D.mt; ++k)
        rows.push_back({xline[k], kind < 2 ? D.h : -D.h, j * d, (kind % 2 == 0) ? 0 : 2});
  std::vector<PxRow> prow_w(rows.begin(), rows.begin() + 4 * D.mw);  // proxies at the walls
  std::vector<PxRow> prow_t(rows.begin() + 4 * D.mw, rows.begin() + 4 * D.mw + 4 * D.mt);  // ... on the lines
  std::vector<double> p4(4 * (size_t)D.mp);
  for (int p = 0; p < D.mp; ++p) {
    const double t = 2.0 * M_PI * p / D.mp;
    p4[4 * p] = rp * std::cos(t);
    p4[4 * p + 1] = rp * std::sin(t);
    p4[4 * p + 2] = std::cos(t);
    p4[4 * p + 3] = std::sin(t);
  }
  std::vector<double> kx(nq), ky(nq);
  for (int i = 0; i < nq; ++i) { kx[i] = omega * std::cos(theta[i]); ky[i] = omega * std::sin(theta[i]); }
  // the angles' columns of f in group order
  std::vector<int> col_of(nq);
  std::vector<PxGroup> pg(ng);
  int64_t s_off = 0, r_off = 0;
  {
    int col = 0;
    for (int g = 0; g < ng; ++g) {
      const std::complex<double> al = std::exp(std::complex<double>(0.0, omega * d * std::cos(theta[groups[g][0]])));
      pg[g].alpha = cmk(al.real(), al.imag());
      pg[g].kap0 = omega * std::cos(theta[groups[g][0]]);
      pg[g].q = (int)groups[g].size();
      pg[g].col0 = col;
      pg[g].s_off = s_off;
      pg[g].r_off = r_off;
      s_off += (int64_t)D.ms * D.ns;
      r_off += (int64_t)D.ms * pg[g].q;
      for (int64_t i : groups[g]) col_of[i] = col++;
    }
  }
  std::vector<double> kxg(nq), kyg(nq);
  for (int i = 0; i < nq; ++i) { kxg[col_of[i]] = kx[i]; kyg[col_of[i]] = ky[i]; }
  D.ycols = l + D.mp + nq;

  const DevGeom g = Handle_geom(h);
  DevBuf<PxRow> drows, dpw, dpt;
  drows.upload(rows, s);
  dpw.upload(prow_w, s);
  dpt.upload(prow_t, s);
  DevBuf<double> dp4, dkx, dky, dxl;
  dp4.upload(p4, s);
  dkx.upload(kxg, s);
  dky.upload(kyg, s);
  dxl.upload(xline, s);
  // 1. row operator (rtot x N): R_{-1}, R_1, then the wall and line rows
  DevBuf<cplx> Rows((size_t)D.rtot * N);
  if (l > 0) {
    HBS_CUDA(cudaMemcpy2DAsync(Rows.get(), sizeof(cplx) * D.rtot, h.Rm.get(), sizeof(cplx) * l, sizeof(cplx) * l, N,
                               cudaMemcpyDeviceToDevice, s));
    HBS_CUDA(cudaMemcpy2DAsync(Rows.get() + l, sizeof(cplx) * D.rtot, h.Rp.get(), sizeof(cplx) * l, sizeof(cplx) * l,
                               N, cudaMemcpyDeviceToDevice, s));
  }
  {
    prof::KScope _ks("k_px_rows", s);
    k_px_rows<<<grid_1d((int64_t)rows.size() * N), 256, 0, s>>>(g, drows.get(), (int)rows.size(), 2 * l, Rows.get(),
                                                               D.rtot);
  }
  HBS_LAUNCH_CHECK("k_px_rows");
  // proxy blocks at the walls (u, u_x at L then R: 4 mw rows) and on the lines (4 mt rows)
  DevBuf<cplx> Qw((size_t)4 * D.mw * D.mp), Vp((size_t)4 * D.mt * D.mp);
  {
    prof::KScope _ks("k_px_proxy_rows", s);
    k_px_proxy_rows<<<grid_1d((int64_t)4 * D.mw * D.mp), 256, 0, s>>>(dpw.get(), 4 * D.mw, dp4.get(), D.mp, omega,
                                                                       Qw.get());
    k_px_proxy_rows<<<grid_1d((int64_t)4 * D.mt * D.mp), 256, 0, s>>>(dpt.get(), 4 * D.mt, dp4.get(), D.mp, omega,
                                                                       Vp.get());
  }
  HBS_LAUNCH_CHECK("k_px_proxy_rows");
  // QL, QR as separate (2 mw x mp) blocks
  DevBuf<cplx> QL((size_t)2 * D.mw * D.mp), QR((size_t)2 * D.mw * D.mp);
  HBS_CUDA(cudaMemcpy2DAsync(QL.get(), sizeof(cplx) * 2 * D.mw, Qw.get(), sizeof(cplx) * 4 * D.mw,
                             sizeof(cplx) * 2 * D.mw, D.mp, cudaMemcpyDeviceToDevice, s));
  HBS_CUDA(cudaMemcpy2DAsync(QR.get(), sizeof(cplx) * 2 * D.mw, Qw.get() + 2 * D.mw, sizeof(cplx) * 4 * D.mw,
                             sizeof(cplx) * 2 * D.mw, D.mp, cudaMemcpyDeviceToDevice, s));
  // 2. X = A^{-1} [P | Phi | f]
  DevBuf<cplx> F((size_t)N * D.ycols), X((size_t)N * D.ycols);
  {
    prof::KScope _ks("k_px_rhs", s);
    k_px_rhs<<<grid_1d(N * D.ycols), 256, 0, s>>>(g, h.Pnb.get(), l, dp4.get(), D.mp, dkx.get(), dky.get(), nq,
                                                  F.get());
  }
  HBS_LAUNCH_CHECK("k_px_rhs");
  h.apply_inverse(F.get(), X.get(), D.ycols, s);
  // 3. Y = Rows X
  DevBuf<cplx> Y((size_t)D.rtot * D.ycols);
  {
    std::vector<GemmJob> gj(1);
    gj[0] = {Rows.get(), X.get(), Y.get(), D.rtot, D.ycols, (int)N, D.rtot, (int)N, D.rtot, cmk(1, 0), cmk(0, 0), 0, 0,
             0, 0, 0};
    run_gemms(gj, s);
  }
  // 4. per Bloch phase: assemble and solve
  DevBuf<PxGroup> dg;
  dg.upload(pg, s);
  DevBuf<cplx> S(std::max<int64_t>(s_off, 1)), Rr(std::max<int64_t>(r_off, 1));
  DevBuf<double> colsc((size_t)ng * D.ns);
  {
    prof::KScope _ks("k_px_assemble", s);
    int qmax = 0;
    for (const auto& gg : pg) qmax = std::max(qmax, gg.q);
    const int64_t per = (int64_t)D.ms * (D.ns + qmax);
    k_px_assemble<<<dim3((unsigned)std::min<int64_t>(1024, (per + 255) / 256), ng), 256, 0, s>>>(
        D, dg.get(), Y.get(), QL.get(), QR.get(), Vp.get(), dxl.get(), S.get(), Rr.get());
  }
  HBS_LAUNCH_CHECK("k_px_assemble");
  {
    prof::KScope _ks("k_px_lsq", s, 8.0 * 2.0 * (double)ng * D.ms * D.ns * D.ns, 0.0);
    k_px_lsq<<<ng, kLsqNT, 0, s>>>(D, dg.get(), S.get(), Rr.get(), colsc.get());
  }
  HBS_LAUNCH_CHECK("k_px_lsq");
  // 5. c_n, d_n at +-y0 and the flux balance of every angle
  std::vector<PxAngle> pa;
  std::vector<int64_t> pa_theta;
  int nout = 0;
  for (int gi = 0; gi < ng; ++gi) {
    const PxGroup& G = pg[gi];
    for (int a = 0; a < G.q; ++a) {
      const int64_t ti = groups[gi][a];
      PxAngle A{};
      A.kap = omega * std::cos(theta[ti]);
      A.k0 = omega * std::fabs(std::sin(theta[ti]));
      A.m = (int)std::llround((A.kap - G.kap0) * d / (2.0 * M_PI));
      A.n_min = (int)std::ceil((-omega - A.kap) * d / (2.0 * M_PI));
      A.n_max = (int)std::floor((omega - A.kap) * d / (2.0 * M_PI));
      A.z_off = G.r_off + (int64_t)a * D.ms;
      A.out_off = nout;
      nout += std::max(0, A.n_max - A.n_min + 1);
      pa.push_back(A);
      pa_theta.push_back(ti);
    }
  }
  DevBuf<PxAngle> dpa;
  dpa.upload(pa, s);
  DevBuf<cplx> cb(std::max(nout, 1)), db(std::max(nout, 1));
  DevBuf<double> fb(pa.size());
  {
    prof::KScope _ks("k_px_bragg", s);
    k_px_bragg<<<(unsigned)pa.size(), 256, 0, s>>>(D, dpa.get(), Rr.get(), h.y0, cb.get(), db.get(), fb.get());
  }
  HBS_LAUNCH_CHECK("k_px_bragg");
  const auto hc = cb.download(s), hd = db.download(s);
  const auto hf = fb.download(s);
  for (size_t t = 0; t < pa.size(); ++t) {
    AngleResult& ar = out.angles[pa_theta[t]];
    ar.n_min = pa[t].n_min;
    ar.n_max = pa[t].n_max;
    for (int n = 0; n <= pa[t].n_max - pa[t].n_min; ++n) {
      ar.c.emplace_back(hc[pa[t].out_off + n].x, hc[pa[t].out_off + n].y);
      ar.d.emplace_back(hd[pa[t].out_off + n].x, hd[pa[t].out_off + n].y);
    }
    ar.flux_err = hf[t];
  }
}

}  // namespace hbs
