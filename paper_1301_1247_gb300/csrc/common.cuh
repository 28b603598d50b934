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

// Boundary geometry, structure-of-arrays on the device.
struct DevGeom {
  const double* x;
  const double* y;
  const double* nx;
  const double* ny;
  const double* w;  // (2 pi / N) |z'(t_j)|
  int64_t n;
  double omega;
  bool df;  // Hankel series in double-float arithmetic (the thread's double-float mode)
};

// Entry A_ij of the Nystrom matrix (Sec. 2.3), including delta_ij / 2.
__device__ __forceinline__ cplx a_entry(const DevGeom& g, int64_t i, int64_t j) {
  if (i == j) return cmk(0.5, 0.0);
  cplx k = combined_kernel(g.x[i], g.y[i], g.x[j], g.y[j], g.nx[j], g.ny[j], g.omega, g.df);
  return cscale(k, kr6_weight(i, j, g.n) * g.w[j]);
}

// Entry of the image block A_s (source obstacle shifted by shift_x): plain trapezoid weights.
__device__ __forceinline__ cplx a_image_entry(const DevGeom& g, int64_t i, int64_t j, double shift_x) {
  cplx k = combined_kernel(g.x[i], g.y[i], g.x[j] + shift_x, g.y[j], g.nx[j], g.ny[j], g.omega, g.df);
  return cscale(k, g.w[j]);
}
