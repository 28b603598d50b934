// Double-float arithmetic: a value is an unevaluated pair of floats (hi, lo), hi + lo,
// with about 48 significant bits.  Products are made error-free with fmaf and sums with
// two-sum, so every operation runs on the FP32 pipes, which GB300 issues at 64 times its
// FP64 rate.  Used for the dense products and the trailing updates of the pivoted QR
// when a handle is built with double-float precision.
#pragma once

#include "common.cuh"

namespace hbs {

// acc += x * y   (double-float, lazy low part; renormalised by df_norm)
// (explicit _rn intrinsics: the compiler may not contract these into FMAs, which would
// break the error-free transformations)
__device__ __forceinline__ void df_mac(float xh, float xl, float yh, float yl, float& ah, float& al) {
  const float p = __fmul_rn(xh, yh);
  float e = fmaf(xh, yh, -p);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  const float sum = __fadd_rn(ah, p);
  const float v = __fsub_rn(sum, ah);
  const float t = __fadd_rn(__fsub_rn(ah, __fsub_rn(sum, v)), __fsub_rn(p, v));
  al = __fadd_rn(al, __fadd_rn(t, e));
  ah = sum;
}
__device__ __forceinline__ void df_norm(float& ah, float& al) {
  const float sum = __fadd_rn(ah, al);
  al = __fsub_rn(al, __fsub_rn(sum, ah));
  ah = sum;
}

// Complex double-float (16 bytes, the size of a complex double, so a complex128 array
// can hold it in place).
struct __align__(16) dfc {
  float rh, rl, ih, il;
};

// Split of an FP64 value into a float pair (hi, lo) with integer operations only (the
// FP64 conversion path shares the scarce FP64 pipe): hi carries the top 24 bits of the
// significand, lo the remainder rounded to 24 bits, so hi + lo equals x to 2^-48
// relative.  Values below the float range become 0.
__device__ __forceinline__ void df_split_bits(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sgn = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const int fe = e - 1023 + 127;
  if (e == 0 || fe < 1) {
    hi = __uint_as_float(sgn);
    lo = __uint_as_float(sgn);
    return;
  }
  if (fe > 254) {
    hi = __uint_as_float(sgn | 0x7f800000u);
    lo = 0.0f;
    return;
  }
  hi = __uint_as_float(sgn | ((unsigned int)fe << 23) | (unsigned int)(m >> 29));
  const unsigned int r = (unsigned int)(m & 0x1FFFFFFFull);  // remainder, r 2^(e-1075)
  if (r == 0u) {
    lo = 0.0f;
    return;
  }
  const int lz = __clz(r) - 3;  // leading zeros within the 29-bit field
  int fel = fe - 24 - lz;
  const unsigned int rn = r << lz;  // leading one at bit 28
  unsigned int q = (rn + 16u) >> 5;  // 24-bit significand, rounded to nearest
  if (q >> 24) {
    q >>= 1;
    ++fel;
  }
  if (fel < 1) {
    lo = 0.0f;
    return;
  }
  lo = __uint_as_float(sgn | ((unsigned int)fel << 23) | (q & 0x7FFFFFu));
}

// float -> double with integer operations only (exact for normal floats; subnormal floats,
// below 1.2e-38, become 0).
__device__ __forceinline__ double f2d_bits(float x) {
  const unsigned int u = __float_as_uint(x);
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0u) return __longlong_as_double((long long)sgn);
  const unsigned long long de = e == 0xFFu ? 0x7FFull : (unsigned long long)(e - 127u + 1023u);
  return __longlong_as_double((long long)(sgn | (de << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

__device__ __forceinline__ dfc to_dfc_bits(cplx v) {
  dfc r;
  df_split_bits(v.x, r.rh, r.rl);
  df_split_bits(v.y, r.ih, r.il);
  return r;
}


// (ah, al) += (bh, bl), lazy low part.
__device__ __forceinline__ void df_add_to(float bh, float bl, float& ah, float& al) {
  const float sum = __fadd_rn(ah, bh);
  const float v = __fsub_rn(sum, ah);
  const float t = __fadd_rn(__fsub_rn(ah, __fsub_rn(sum, v)), __fsub_rn(bh, v));
  al = __fadd_rn(al, __fadd_rn(t, bl));
  ah = sum;
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

__device__ __forceinline__ dfc dfc_shfl_xor(const dfc& a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.rh, o), __shfl_xor_sync(0xffffffffu, a.rl, o),
          __shfl_xor_sync(0xffffffffu, a.ih, o), __shfl_xor_sync(0xffffffffu, a.il, o)};
}

__device__ __forceinline__ dfc dfc_shfl(const dfc& a, int l) {
  return {__shfl_sync(0xffffffffu, a.rh, l), __shfl_sync(0xffffffffu, a.rl, l), __shfl_sync(0xffffffffu, a.ih, l),
          __shfl_sync(0xffffffffu, a.il, l)};
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
