// Double-float arithmetic: a value is an unevaluated pair of floats (hi, lo), hi + lo,
// with about 48 significant bits.  Products are made error-free with fmaf and sums with
// two-sum, so every operation runs on the FP32 pipes, which GB300 issues at 64 times its
// FP64 rate.  Used for the dense products and the trailing updates of the pivoted QR
// when a handle is built with double-float precision.
#pragma once

#include "common.cuh"
#include "dfcore.cuh"

namespace hbs {

// Complex double-float (16 bytes, the size of a complex double, so a complex128 array
// can hold it in place).
struct __align__(16) dfc {
  float rh, rl, ih, il;
};

__device__ __forceinline__ dfc to_dfc_bits(cplx v) {
  dfc r;
  df_split_bits(v.x, r.rh, r.rl);
  df_split_bits(v.y, r.ih, r.il);
  return r;
}


__device__ __forceinline__ cplx from_dfc_bits(const dfc& v) {
  return cmk(f2d_bits(v.rh) + f2d_bits(v.rl), f2d_bits(v.ih) + f2d_bits(v.il));
}

__device__ __forceinline__ void dfc_norm(dfc& a) {
  df_norm(a.rh, a.rl);
  df_norm(a.ih, a.il);
}

// acc += conj(v) a   (lazy low parts)
__device__ __forceinline__ void dfc_cdot_acc(const dfc& v, const dfc& a, dfc& acc) {
  df_mac(v.rh, v.rl, a.rh, a.rl, acc.rh, acc.rl);
  df_mac(v.ih, v.il, a.ih, a.il, acc.rh, acc.rl);
  df_mac(v.rh, v.rl, a.ih, a.il, acc.ih, acc.il);
  df_mac(-v.ih, -v.il, a.rh, a.rl, acc.ih, acc.il);
}

// a -= v w   (renormalised)
__device__ __forceinline__ void dfc_sub_mul(const dfc& v, const dfc& w, dfc& a) {
  df_mac(-v.rh, -v.rl, w.rh, w.rl, a.rh, a.rl);
  df_mac(v.ih, v.il, w.ih, w.il, a.rh, a.rl);
  df_mac(-v.rh, -v.rl, w.ih, w.il, a.ih, a.il);
  df_mac(-v.ih, -v.il, w.rh, w.rl, a.ih, a.il);
  dfc_norm(a);
}

// a b   (renormalised)
__device__ __forceinline__ dfc dfc_mul(const dfc& a, const dfc& b) {
  dfc r{0.f, 0.f, 0.f, 0.f};
  df_mac(a.rh, a.rl, b.rh, b.rl, r.rh, r.rl);
  df_mac(-a.ih, -a.il, b.ih, b.il, r.rh, r.rl);
  df_mac(a.rh, a.rl, b.ih, b.il, r.ih, r.il);
  df_mac(a.ih, a.il, b.rh, b.rl, r.ih, r.il);
  dfc_norm(r);
  return r;
}

// acc += |a|^2   (lazy low part)
__device__ __forceinline__ void df_abs2_acc(const dfc& a, float& ah, float& al) {
  df_mac(a.rh, a.rl, a.rh, a.rl, ah, al);
  df_mac(a.ih, a.il, a.ih, a.il, ah, al);
}

// s * a for a double-float real s = (sh, sl)   (renormalised)
__device__ __forceinline__ dfc dfc_scale(float sh, float sl, const dfc& a) {
  dfc r{0.f, 0.f, 0.f, 0.f};
  df_mac(sh, sl, a.rh, a.rl, r.rh, r.rl);
  df_mac(sh, sl, a.ih, a.il, r.ih, r.il);
  dfc_norm(r);
  return r;
}

// 1 / d = conj(d) / |d|^2 (0 for d = 0)
__device__ __forceinline__ dfc dfc_recip(const dfc& d) {
  float nh = 0.f, nl = 0.f;
  df_abs2_acc(d, nh, nl);
  df_norm(nh, nl);
  if (!(nh > 0.f)) return {0.f, 0.f, 0.f, 0.f};
  float qh, ql;
  df_div(1.f, 0.f, nh, nl, qh, ql);
  const dfc c{d.rh, d.rl, -d.ih, -d.il};
  return dfc_scale(qh, ql, c);
}

__device__ __forceinline__ dfc dfc_shfl_xor(const dfc& a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.rh, o), __shfl_xor_sync(0xffffffffu, a.rl, o),
          __shfl_xor_sync(0xffffffffu, a.ih, o), __shfl_xor_sync(0xffffffffu, a.il, o)};
}

__device__ __forceinline__ dfc dfc_shfl(const dfc& a, int l) {
  return {__shfl_sync(0xffffffffu, a.rh, l), __shfl_sync(0xffffffffu, a.rl, l), __shfl_sync(0xffffffffu, a.ih, l),
          __shfl_sync(0xffffffffu, a.il, l)};
}

// The Householder reflector of x = (x0, x_1, ...) in double-float arithmetic (the FP64
// formulas of householder_scalars, with ||x_1..||^2 = sig): beta = -(x0/|x0|) ||x||,
// v0 = x0 - beta, tau = 2 / (|v0|^2 + sig).  One thread, FP32 pipes only.
__device__ __forceinline__ void df_householder(const dfc& x0, float sh, float sl, dfc* v0, dfc* beta, float* th,
                                               float* tl) {
  float a2h = 0.f, a2l = 0.f;
  df_abs2_acc(x0, a2h, a2l);
  df_norm(a2h, a2l);
  float axh, axl;
  df_sqrt(a2h, a2l, axh, axl);
  float t2h = a2h, t2l = a2l;
  df_add_to(sh, sl, t2h, t2l);
  df_norm(t2h, t2l);
  float xnh, xnl;
  df_sqrt(t2h, t2l, xnh, xnl);
  dfc v, b;
  if (axh > 0.f) {
    float fh, fl;  // ||x|| / |x0|
    df_div(xnh, xnl, axh, axl, fh, fl);
    b = dfc_scale(-fh, -fl, x0);
    v = x0;  // x0 (1 + f)
    df_mac(x0.rh, x0.rl, fh, fl, v.rh, v.rl);
    df_mac(x0.ih, x0.il, fh, fl, v.ih, v.il);
    dfc_norm(v);
  } else {
    b = {-xnh, -xnl, 0.f, 0.f};
    v = {xnh, xnl, 0.f, 0.f};
  }
  float vvh = 0.f, vvl = 0.f;
  df_abs2_acc(v, vvh, vvl);
  df_add_to(sh, sl, vvh, vvl);
  df_norm(vvh, vvl);
  if (vvh > 0.f) {
    df_div(2.f, 0.f, vvh, vvl, *th, *tl);
  } else {
    *th = 0.f;
    *tl = 0.f;
  }
  *v0 = v;
  *beta = b;
}

// Block-wide double-float sum formed in warp 0 (red: 2 NT floats).  The result is valid
// in every lane of warp 0.  Contains one __syncthreads.
template <int NT>
__device__ __forceinline__ void block_sum_df_warp0(float& h, float& l, float* red) {
  red[threadIdx.x] = h;
  red[NT + threadIdx.x] = l;
  __syncthreads();
  if (threadIdx.x < 32) {
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) df_add_to(red[threadIdx.x + 32 * k], red[NT + threadIdx.x + 32 * k], sh, sl);
    df_norm(sh, sl);
    for (int o = 16; o > 0; o >>= 1) {
      const float bh = __shfl_xor_sync(0xffffffffu, sh, o), bl = __shfl_xor_sync(0xffffffffu, sl, o);
      df_add_to(bh, bl, sh, sl);
    }
    df_norm(sh, sl);
    h = sh;
    l = sl;
  }
}

// Warp sum of a complex double-float value; every lane receives lane 0's result.
__device__ __forceinline__ dfc dfc_warp_sum(dfc a) {
  dfc_norm(a);
  for (int o = 16; o > 0; o >>= 1) {
    const dfc b = dfc_shfl_xor(a, o);
    df_add_to(b.rh, b.rl, a.rh, a.rl);
    df_add_to(b.ih, b.il, a.ih, a.il);
  }
  dfc_norm(a);
  return dfc_shfl(a, 0);
}

}  // namespace hbs
