// Scalar double-float arithmetic: a value is an unevaluated pair of floats (hi, lo),
// hi + lo, with about 48 significant bits.  Products are made error-free with fmaf and
// sums with two-sum, so every operation runs on the FP32 pipes, which GB300 issues at 64
// times its FP64 rate.  Conversions to and from FP64 use integer operations only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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

// (ah, al) += (bh, bl), lazy low part.
__device__ __forceinline__ void df_add_to(float bh, float bl, float& ah, float& al) {
  const float sum = __fadd_rn(ah, bh);
  const float v = __fsub_rn(sum, ah);
  const float t = __fadd_rn(__fsub_rn(ah, __fsub_rn(sum, v)), __fsub_rn(bh, v));
  al = __fadd_rn(al, __fadd_rn(t, bl));
  ah = sum;
}

// Double-float square root of a = (ah, al) >= 0: sqrtf of the high part and one Newton
// correction (a - y^2 is exact for y = RN(sqrt(ah)), via fmaf).
__device__ __forceinline__ void df_sqrt(float ah, float al, float& rh, float& rl) {
  if (!(ah > 0.f)) {
    rh = 0.f;
    rl = 0.f;
    return;
  }
  const float y = sqrtf(ah);
  const float e = fmaf(-y, y, ah);
  const float c = __fdiv_rn(__fadd_rn(e, al), __fmul_rn(2.f, y));
  rh = __fadd_rn(y, c);
  rl = __fsub_rn(c, __fsub_rn(rh, y));
}

// Double-float quotient a / b: q1 = ah / bh and one correction from the remainder
// a - q1 b (q1 bh error-free via fmaf).
__device__ __forceinline__ void df_div(float ah, float al, float bh, float bl, float& qh, float& ql) {
  const float q1 = __fdiv_rn(ah, bh);
  const float p = __fmul_rn(q1, bh);
  const float pe = fmaf(q1, bh, -p);
  const float r = __fadd_rn(__fsub_rn(ah, p), __fsub_rn(__fsub_rn(al, pe), __fmul_rn(q1, bl)));
  const float q2 = __fdiv_rn(r, bh);
  qh = __fadd_rn(q1, q2);
  ql = __fsub_rn(q2, __fsub_rn(qh, q1));
}

}  // namespace hbs
