// Double-float device helpers (pairs of FP32 numbers standing for one FP64
// value; see df.cu for the scheme and its error bounds), shared by the
// double-float product (df.cu) and the double-float Arnoldi process
// (krylov.cu).
#pragma once
#include <cuda_runtime.h>

namespace hz {

// Conversions between FP64 and double-float by the IEEE-754 bit layouts, so
// that they issue integer instructions instead of FP64-pipe conversions.
//
// x -> (hi, lo): hi keeps the sign, exponent and leading 24 significant bits
// of x (truncated); lo is the remaining 29 bits rounded to 23, built from its
// bits as (1 + r) 2^(E-23) - 2^(E-23) (one exact FP32 subtraction), so that
// |hi + lo - x| <= 2^-47 |x|. Zeros and FP64 subnormals give (0, 0); values
// outside [2^-103, 2^128) fall back to one rounding (lo = 0).
static __device__ __forceinline__ float2 df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return make_float2(__uint_as_float(sign), 0.f);
  const int fe = e - 1023 + 127;
  if (fe <= 23 || fe >= 255) return make_float2(__double2float_rn(x), 0.f);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)(m >> 29));
  const unsigned base = (unsigned)(fe - 23) << 23;                        // 2^(E-23) as FP32 bits
  const unsigned r23 = (unsigned)(((m & 0x1FFFFFFFull) + 32ull) >> 6);      // rounded, may carry to 2^23
  const float lo = __fsub_rn(__uint_as_float(base + r23), __uint_as_float(base));
  return make_float2(hi, sign ? -lo : lo);
}

// FP32 -> FP64 (exact)
static __device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if ((u & 0x7FFFFFFFu) == 0) return __longlong_as_double((long long)sign);
  if (e == 0 || e == 255) return (double)f;  // subnormal, inf, nan
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// (sh, sl) += (ah + al) (xh + xl); the al*xl term (2^-48 relative) is dropped
static __device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float xh, float xl) {
  const float p = __fmul_rn(ah, xh);
  float e = __fmaf_rn(ah, xh, -p);  // exact: ah*xh = p + e
  e = __fmaf_rn(ah, xl, e);
  e = __fmaf_rn(al, xh, e);
  const float t = __fadd_rn(sh, p);  // TwoSum: sh + p = t + err exactly
  const float z = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
  sl = __fadd_rn(sl, __fadd_rn(err, e));
  sh = t;
}

// renormalise (h, l) so that |l| is at most half an ulp of h (Fast2Sum; |h| >= |l| or h = 0)
static __device__ __forceinline__ void df_norm(float& h, float& l) {
  const float t = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(t, h));
  h = t;
}

// (h, l) = (ah + al) (bh + bl), renormalised; the al*bl term is dropped
static __device__ __forceinline__ void df_mul(float& h, float& l, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  h = p;
  l = e;
  df_norm(h, l);
}

}  // namespace hz
