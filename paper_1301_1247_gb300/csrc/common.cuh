// Shared device helpers: complex FP64 arithmetic, Hankel functions H0^(1), H1^(1),
// and the combined-field kernel of the Nystrom matrix (Sec. 2.2-2.3).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dfcore.cuh"
#include "hankel_table.h"

typedef double2 cplx;

__host__ __device__ __forceinline__ cplx cmk(double re, double im) { return make_double2(re, im); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return cmk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ cplx cscale(cplx a, double s) { return cmk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return cmk(a.x, -a.y); }
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double cabs1(cplx a) { return sqrt(a.x * a.x + a.y * a.y); }
// acc += a * b
__host__ __device__ __forceinline__ cplx cfma(cplx a, cplx b, cplx acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc - a * b, four fused multiply-adds
__host__ __device__ __forceinline__ cplx cfms(cplx a, cplx b, cplx acc) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  // Smith's algorithm
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, den = b.x + b.y * r;
    return cmk((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  } else {
    double r = b.x / b.y, den = b.x * r + b.y;
    return cmk((a.x * r + a.y) / den, (a.y * r - a.x) / den);
  }
}
__device__ __forceinline__ cplx cexp_i(double t) {  // exp(i t)
  double s, c;
  sincos(t, &s, &c);
  return cmk(c, s);
}
__device__ __forceinline__ cplx cexp(cplx z) {  // exp(z)
  double e = exp(z.x), s, c;
  sincos(z.y, &s, &c);
  return cmk(e * c, e * s);
}
__device__ __forceinline__ cplx csqrt_principal(cplx z) {
  double r = hypot(z.x, z.y);
  if (r == 0.0) return cmk(0.0, 0.0);
  double t = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return cmk(t, z.y / (2.0 * t));
  return cmk(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

#define HBS_PI 3.14159265358979323846
#define HBS_EULER_GAMMA 0.57721566490153286061

// ---------------------------------------------------------------------------
// Hankel functions of the first kind, orders 0 and 1, real argument z > 0.
//
// z < 40: piecewise Chebyshev expansions (hankel_table.h, intervals of width 1/2, 11 terms) of
//   J0, J1 and, below z = 4, of the regular parts of Neumann's expansions,
//     R0 = Y0 - (2/pi)(ln(z/2) + gamma) J0,   R1 = Y1 - (2/pi)(ln(z/2) + gamma) J1 + 2/(pi z),
//   so that Y0 and Y1 take one logarithm; from z = 4 on, of Y0 and Y1 themselves.  The four
//   series are summed together by Clenshaw's recurrence, in FP64 or (df) in double-float
//   arithmetic on the FP32 pipes.
// z >= 40: Hankel's asymptotic expansion
//     H_nu(z) ~ sqrt(2/(pi z)) e^{i(z - nu pi/2 - pi/4)} sum_k i^k a_k(nu) / z^k,
//     a_k(nu) = a_{k-1}(nu) (4 nu^2 - (2k-1)^2) / (8k),
//   summed until the term falls below 1e-17 (at most 48 terms).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void hankel01(double z, cplx* h0, cplx* h1, bool df = false) {
  if (z < (double)(kHankelIntervals / kHankelPerUnit)) {
    const double zp = (double)kHankelPerUnit * z;  // exact (power of two)
    const int iv = (int)zp;
    const double t = 2.0 * (zp - (double)iv) - 1.0;
    double v[4];
    if (df) {
      // Clenshaw in double-float arithmetic (FP32 pipes, about 2^-48 per operation)
      float th, tl;
      hbs::df_split_bits(t, th, tl);
      const float t2h = 2.0f * th, t2l = 2.0f * tl;
      const float* c = kHankelChebDF + (size_t)iv * 8 * kHankelDegree;
      float b1h[4] = {0.f, 0.f, 0.f, 0.f}, b1l[4] = {0.f, 0.f, 0.f, 0.f};
      float b2h[4] = {0.f, 0.f, 0.f, 0.f}, b2l[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = kHankelDegree - 1; k >= 1; --k) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          float bh = __ldg(c + 2 * (f * kHankelDegree + k)), bl = __ldg(c + 2 * (f * kHankelDegree + k) + 1);
          hbs::df_add_to(-b2h[f], -b2l[f], bh, bl);
          hbs::df_mac(t2h, t2l, b1h[f], b1l[f], bh, bl);
          hbs::df_norm(bh, bl);
          b2h[f] = b1h[f];
          b2l[f] = b1l[f];
          b1h[f] = bh;
          b1l[f] = bl;
        }
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        float bh = __ldg(c + 2 * f * kHankelDegree), bl = __ldg(c + 2 * f * kHankelDegree + 1);
        hbs::df_add_to(-b2h[f], -b2l[f], bh, bl);
        hbs::df_mac(th, tl, b1h[f], b1l[f], bh, bl);
        v[f] = hbs::f2d_bits(bh) + hbs::f2d_bits(bl);
      }
    } else {
      const double t2 = 2.0 * t;
      const double* c = kHankelCheb + (size_t)iv * 4 * kHankelDegree;
      double b1[4] = {0.0, 0.0, 0.0, 0.0}, b2[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int k = kHankelDegree - 1; k >= 1; --k) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const double b0 = fma(t2, b1[f], __ldg(c + f * kHankelDegree + k) - b2[f]);
          b2[f] = b1[f];
          b1[f] = b0;
        }
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) v[f] = fma(t, b1[f], __ldg(c + f * kHankelDegree) - b2[f]);
    }
    if (iv >= kHankelDirect) {  // Y0, Y1 tabulated directly
      *h0 = cmk(v[0], v[2]);
      *h1 = cmk(v[1], v[3]);
    } else {
      const double lg = (2.0 / HBS_PI) * (log(0.5 * z) + HBS_EULER_GAMMA);
      *h0 = cmk(v[0], fma(lg, v[0], v[2]));
      *h1 = cmk(v[1], fma(lg, v[1], v[3]) - 2.0 / (HBS_PI * z));
    }
  } else {
    // unrolled: the ratios (4 nu^2 - (2k-1)^2) / (8k) are literals
    const double iz = 1.0 / z;
    double a0 = 1.0, a1 = 1.0, p = 1.0;
    double s0r = 1.0, s0i = 0.0, s1r = 1.0, s1i = 0.0;
#pragma unroll
    for (int k = 1; k < 48; ++k) {
      const double q = (double)(2 * k - 1);
      a0 *= (0.0 - q * q) / (8.0 * k);
      a1 *= (4.0 - q * q) / (8.0 * k);
      p *= iz;
      const double t0 = a0 * p, t1 = a1 * p;
      switch (k & 3) {
        case 0: s0r += t0; s1r += t1; break;
        case 1: s0i += t0; s1i += t1; break;
        case 2: s0r -= t0; s1r -= t1; break;
        default: s0i -= t0; s1i -= t1; break;
      }
      if (fabs(t0) < 1e-17 && fabs(t1) < 1e-17) break;
    }
    double amp = sqrt(2.0 / (HBS_PI * z));
    double sn, cs;
    sincos(z - 0.25 * HBS_PI, &sn, &cs);  // chi_0
    // e^{i chi_1} = e^{i chi_0} e^{-i pi/2} = -i e^{i chi_0}
    cplx e0 = cmk(amp * cs, amp * sn);
    cplx e1 = cmk(amp * sn, -amp * cs);
    *h0 = cmul(e0, cmk(s0r, s0i));
    *h1 = cmul(e1, cmk(s1r, s1i));
  }
}

// i c H1 + (w/4) H0: the combined-field kernel once the geometric factor
// c = (w/4) ((x - y).n_y) / r is known.
__device__ __forceinline__ cplx combined_from(double c, cplx h0, cplx h1, double omega) {
  return cmk(-c * h1.y + 0.25 * omega * h0.x, c * h1.x + 0.25 * omega * h0.y);
}

// Combined-field kernel dG/dn_y - i w G at target (tx, ty), source (sx, sy) with unit
// normal (nx, ny), G = (i/4) H0(w r):  (i w / 4) H1(w r) ((x - y).n_y) / r + (w / 4) H0(w r).
__device__ __forceinline__ cplx combined_kernel(double tx, double ty, double sx, double sy,
                                                double nx, double ny, double omega, bool df = false) {
  double dx = tx - sx, dy = ty - sy;
  double r = sqrt(dx * dx + dy * dy);
  cplx h0, h1;
  hankel01(omega * r, &h0, &h1, df);
  double c = 0.25 * omega * (dx * nx + dy * ny) / r;
  // i c H1 + (w/4) H0
  return cmk(-c * h1.y + 0.25 * omega * h0.x, c * h1.x + 0.25 * omega * h0.y);
}

// Single-layer and double-layer kernels used by proxy sources:
// G = (i/4) H0(w r), dG/dn_p = (i w / 4) H1(w r) ((x - p).n_p) / r.
__device__ __forceinline__ void proxy_kernels(double tx, double ty, double px, double py, double nx,
                                              double ny, double omega, cplx* g, cplx* dg, bool df = false) {
  double dx = tx - px, dy = ty - py;
  double r = sqrt(dx * dx + dy * dy);
  cplx h0, h1;
  hankel01(omega * r, &h0, &h1, df);
  *g = cmk(-0.25 * h0.y, 0.25 * h0.x);
  double c = 0.25 * omega * (dx * nx + dy * ny) / r;
  *dg = cmk(-c * h1.y, c * h1.x);
}

// Kapur-Rokhlin 6th-order corrected weights R_j = 1 + gamma_j (j = 1..6), from the
// published table of Kapur & Rokhlin (1997), Table 6, log-singular, order 6 (Sec. 2.3).
__device__ __forceinline__ double kr6_weight(int64_t i, int64_t j, int64_t n) {
  int64_t dd = i > j ? i - j : j - i;
  if (n - dd < dd) dd = n - dd;
  switch (dd) {
    case 0: return 0.0;
    case 1: return 1.0 + 4.967362978287758;
    case 2: return 1.0 - 16.20501504859126;
    case 3: return 1.0 + 25.85153761832639;
    case 4: return 1.0 - 22.22599466791883;
    case 5: return 1.0 + 9.930104998037539;
    case 6: return 1.0 - 1.817995878141594;
    default: return 1.0;
  }
}

// Boundary geometry, structure-of-arrays on the device, indexed by unknown.
//
// Sound-soft obstacles (Sec. 2): one unknown per boundary node.  Transmission problem
// (Sec. 5): two unknowns per node, interlaced: unknown 2p is s_p, the single-layer density
// sigma_p = w s_p in units of w, unknown 2p + 1 the double-layer density tau_p, and row 2p
// (2p + 1) the sigma (tau) row of node p.  Carrying w with the single layer and 1/w with
// the sigma row (a diagonal similarity) balances the 2 x 2 blocks of the operator.  The
// arrays hold every node twice, at both of its unknowns, so that the tree, the near lists
// and every index set of the method address unknowns.
struct DevGeom {
  const double* x;
  const double* y;
  const double* nx;
  const double* ny;
  const double* w;  // (2 pi / N_nodes) |z'(t_j)|
  int64_t n;        // unknowns
  double omega;
  bool df;          // Hankel series in double-float arithmetic (the thread's double-float mode)
  int comps;        // unknowns per node: 1 (sound-soft) or 2 (transmission)
  double omega_in;  // n omega, the wavenumber inside the obstacles (transmission)
};

// Field of a unit source of the single layer (c = 0: G = (i/4) H0(k r)) or of the double
// layer (c = 1: dG/dn_y = (i k/4) H1(k r) (d.n_y)/r) at offset d = x - y (|d| = r), with
// H0, H1 at k r given, and its gradient in the target x:
//   grad G       = -(i k/4) H1 d / r,
//   grad dG/dn_y = (i k/4) [k H0 d (d.n_y)/r^2 + (H1/r) (n_y - 2 d (d.n_y)/r^2)]
// (from H1' = H0 - H1/z).
__device__ __forceinline__ void layer_field(double ddx, double ddy, double r, cplx h0, cplx h1, double k, double snx,
                                            double sny, int c, cplx* v, cplx* gx, cplx* gy) {
  const double ir = 1.0 / r;
  const cplx ik4h1 = cmk(-0.25 * k * h1.y, 0.25 * k * h1.x);  // (i k / 4) H1
  if (c == 0) {
    *v = cmk(-0.25 * h0.y, 0.25 * h0.x);
    *gx = cscale(ik4h1, -ddx * ir);
    *gy = cscale(ik4h1, -ddy * ir);
    return;
  }
  const double cy = (ddx * snx + ddy * sny) * ir;
  *v = cscale(ik4h1, cy);
  const cplx a = cscale(cmk(-0.25 * k * k * h0.y, 0.25 * k * k * h0.x), cy * ir);  // multiplies d
  const cplx b = cscale(ik4h1, ir);
  *gx = cadd(cscale(a, ddx), cscale(b, snx - 2.0 * ddx * cy * ir));
  *gy = cadd(cscale(a, ddy), cscale(b, sny - 2.0 * ddy * cy * ir));
}

// Row functional of the transmission rows (Sec. 5): the tau row of a node takes the value
// of a field, the sigma row minus its normal derivative divided by w.
__device__ __forceinline__ cplx row_functional(const DevGeom& g, int64_t i, cplx v, cplx gx, cplx gy) {
  if (i & 1) return v;
  const double f = -1.0 / g.omega;
  return cmk(f * (g.nx[i] * gx.x + g.ny[i] * gy.x), f * (g.nx[i] * gx.y + g.ny[i] * gy.y));
}

// Transmission: the row of unknown i applied to the source of unknown j placed at
// (sx, sy), wavenumber k, without quadrature weight (single-layer sources carry w).
__device__ __forceinline__ cplx pair_entry(const DevGeom& g, int64_t i, double sx, double sy, int64_t j, double k) {
  const double ddx = g.x[i] - sx, ddy = g.y[i] - sy;
  const double r = sqrt(ddx * ddx + ddy * ddy);
  cplx h0, h1, v, gx, gy;
  hankel01(k * r, &h0, &h1, g.df);
  layer_field(ddx, ddy, r, h0, h1, k, g.nx[j], g.ny[j], (int)(j & 1), &v, &gx, &gy);
  if (!(j & 1)) {
    v = cscale(v, g.omega);
    gx = cscale(gx, g.omega);
    gy = cscale(gy, g.omega);
  }
  return row_functional(g, i, v, gx, gy);
}

// Transmission entry A_ij (Sec. 5): the identity on the node's own 2 x 2 block, else the
// row functional of the outside source minus that of the inside source (the jumps of the
// matching conditions), with the Kapur-Rokhlin weights of the node distance.
__device__ __forceinline__ cplx tr_a_entry(const DevGeom& g, int64_t i, int64_t j) {
  const int64_t p = i >> 1, q = j >> 1;
  if (p == q) return cmk(i == j ? 1.0 : 0.0, 0.0);
  const cplx vo = pair_entry(g, i, g.x[j], g.y[j], j, g.omega);
  const cplx vi = pair_entry(g, i, g.x[j], g.y[j], j, g.omega_in);
  return cscale(csub(vo, vi), kr6_weight(p, q, g.n >> 1) * g.w[j]);
}

// Transmission: A_ij and A_ji together (i, j on different nodes): both share the distance,
// so one Hankel pair per wavenumber serves the two entries.
__device__ __forceinline__ void tr_a_entry_pair(const DevGeom& g, int64_t i, int64_t j, cplx* aij, cplx* aji) {
  const double ddx = g.x[i] - g.x[j], ddy = g.y[i] - g.y[j];
  const double r = sqrt(ddx * ddx + ddy * ddy);
  cplx e_ij = cmk(0.0, 0.0), e_ji = cmk(0.0, 0.0);
  for (int side = 0; side < 2; ++side) {  // outside minus inside
    const double k = side == 0 ? g.omega : g.omega_in;
    cplx h0, h1, v, gx, gy;
    hankel01(k * r, &h0, &h1, g.df);
    // source j seen from i (offset x_i - x_j), source i seen from j (the opposite offset)
    layer_field(ddx, ddy, r, h0, h1, k, g.nx[j], g.ny[j], (int)(j & 1), &v, &gx, &gy);
    if (!(j & 1)) { v = cscale(v, g.omega); gx = cscale(gx, g.omega); gy = cscale(gy, g.omega); }
    const cplx a = row_functional(g, i, v, gx, gy);
    layer_field(-ddx, -ddy, r, h0, h1, k, g.nx[i], g.ny[i], (int)(i & 1), &v, &gx, &gy);
    if (!(i & 1)) { v = cscale(v, g.omega); gx = cscale(gx, g.omega); gy = cscale(gy, g.omega); }
    const cplx b = row_functional(g, j, v, gx, gy);
    e_ij = side == 0 ? a : csub(e_ij, a);
    e_ji = side == 0 ? b : csub(e_ji, b);
  }
  const double kw = kr6_weight(i >> 1, j >> 1, g.n >> 1);
  *aij = cscale(e_ij, kw * g.w[j]);
  *aji = cscale(e_ji, kw * g.w[i]);
}

// Entry A_ij of the Nystrom matrix (Sec. 2.3), including delta_ij / 2.
__device__ __forceinline__ cplx a_entry(const DevGeom& g, int64_t i, int64_t j) {
  if (g.comps == 2) return tr_a_entry(g, i, j);
  if (i == j) return cmk(0.5, 0.0);
  cplx k = combined_kernel(g.x[i], g.y[i], g.x[j], g.y[j], g.nx[j], g.ny[j], g.omega, g.df);
  return cscale(k, kr6_weight(i, j, g.n) * g.w[j]);
}

// Entry of the image block A_s (source obstacle shifted by shift_x): plain trapezoid weights.
__device__ __forceinline__ cplx a_image_entry(const DevGeom& g, int64_t i, int64_t j, double shift_x) {
  if (g.comps == 2) return cscale(pair_entry(g, i, g.x[j] + shift_x, g.y[j], j, g.omega), g.w[j]);
  cplx k = combined_kernel(g.x[i], g.y[i], g.x[j] + shift_x, g.y[j], g.nx[j], g.ny[j], g.omega, g.df);
  return cscale(k, g.w[j]);
}

// Transmission: field (what = 0), x-derivative (1) or y-derivative (2) at a point
// (tx, ty) off the boundary of the layer of unknown j placed at (sx, sy), outside
// wavenumber, without weight (single-layer sources carry w).
__device__ __forceinline__ cplx pair_source_field(const DevGeom& g, double tx, double ty, double sx, double sy,
                                                  int64_t j, int what) {
  const double ddx = tx - sx, ddy = ty - sy;
  const double r = sqrt(ddx * ddx + ddy * ddy);
  cplx h0, h1, v, gx, gy;
  hankel01(g.omega * r, &h0, &h1, g.df);
  layer_field(ddx, ddy, r, h0, h1, g.omega, g.nx[j], g.ny[j], (int)(j & 1), &v, &gx, &gy);
  const cplx out = what == 0 ? v : (what == 1 ? gx : gy);
  return (j & 1) ? out : cscale(out, g.omega);
}

// Transmission: row functional of unknown i applied to a combined-layer proxy source
// dG/dn_p - i k G at (px, py) with normal (pnx, pny), wavenumber k.
__device__ __forceinline__ cplx proxy_row_entry(const DevGeom& g, int64_t i, double px, double py, double pnx,
                                                double pny, double k) {
  const double ddx = g.x[i] - px, ddy = g.y[i] - py;
  const double r = sqrt(ddx * ddx + ddy * ddy);
  cplx h0, h1, v1, gx1, gy1, v0, gx0, gy0;
  hankel01(k * r, &h0, &h1, g.df);
  layer_field(ddx, ddy, r, h0, h1, k, pnx, pny, 1, &v1, &gx1, &gy1);
  layer_field(ddx, ddy, r, h0, h1, k, pnx, pny, 0, &v0, &gx0, &gy0);
  const cplx mik = cmk(0.0, -k);
  return row_functional(g, i, cadd(v1, cmul(mik, v0)), cadd(gx1, cmul(mik, gx0)), cadd(gy1, cmul(mik, gy0)));
}

// Transmission: value at (tx, ty) of the layer of unknown j (at its node), wavenumber k,
// without weight (single-layer sources carry w).
__device__ __forceinline__ cplx layer_value_at(const DevGeom& g, double tx, double ty, int64_t j, double k) {
  const double ddx = tx - g.x[j], ddy = ty - g.y[j];
  const double r = sqrt(ddx * ddx + ddy * ddy);
  cplx h0, h1, v, gx, gy;
  hankel01(k * r, &h0, &h1, g.df);
  layer_field(ddx, ddy, r, h0, h1, k, g.nx[j], g.ny[j], (int)(j & 1), &v, &gx, &gy);
  return (j & 1) ? v : cscale(v, g.omega);
}

// Transmission: for node unknown j and a proxy point p (normal (pnx, pny)) at wavenumber
// k, both proxy rows of the node ID from one Hankel pair: the row functional of j applied
// to the combined-layer proxy source, and the field at p of unknown j's layer.
__device__ __forceinline__ void proxy_pair_entries(const DevGeom& g, int64_t j, double px, double py, double pnx,
                                                   double pny, double k, cplx* row, cplx* field) {
  const double ddx = g.x[j] - px, ddy = g.y[j] - py;
  const double r = sqrt(ddx * ddx + ddy * ddy);
  cplx h0, h1, v1, gx1, gy1, v0, gx0, gy0;
  hankel01(k * r, &h0, &h1, g.df);
  layer_field(ddx, ddy, r, h0, h1, k, pnx, pny, 1, &v1, &gx1, &gy1);
  layer_field(ddx, ddy, r, h0, h1, k, pnx, pny, 0, &v0, &gx0, &gy0);
  const cplx mik = cmk(0.0, -k);
  *row = row_functional(g, j, cadd(v1, cmul(mik, v0)), cadd(gx1, cmul(mik, gx0)), cadd(gy1, cmul(mik, gy0)));
  cplx v, gx, gy;
  layer_field(-ddx, -ddy, r, h0, h1, k, g.nx[j], g.ny[j], (int)(j & 1), &v, &gx, &gy);
  *field = (j & 1) ? v : cscale(v, g.omega);
}
