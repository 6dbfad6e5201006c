// Double-float arithmetic of the outer Krylov basis.
//
// A real value is the unevaluated sum hi + lo of two binary32 numbers with |lo| below
// one unit in the last place of hi; a complex basis value is stored as the float4
// {re.hi, re.lo, im.hi, im.lo}, the same 16 bytes as a complex128.  Products and sums
// run on the FP32 pipe with error-free transformations: the product of two binary32
// numbers is p + e exactly with e = fma(a, b, -p) (Dekker's TwoProduct, formed by one
// FMA), and the sum of two is t + r exactly with Knuth's TwoSum (six additions, no
// branch).  T. J. Dekker, "A floating-point technique for extending the available
// precision", Numer. Math. 18 (1971); D. E. Knuth, TAOCP vol. 2, Sec. 4.2.2.
//
// Accuracy: a double-float here carries 47 significant bits (hi 24, lo 23; a binary64
// value is truncated when split, relative error below 2^-46).  A product of two carries
// a relative error of about 2^-44 (both splits, the dropped lo x lo term, two FMA
// roundings), and a sum of K products accumulated with df_mac and renormalised after
// every term errs by about (4 + K) 2^-45 times the sum of the products' magnitudes:
// the error bound of recursive summation with unit 2^-45 in place of binary64's 2^-53.
// On this part the FP64 pipe issues one instruction where the FP32 pipe issues 64, so
// the twelve FP32 instructions of one multiply-add cost about a fifth of one FP64 FMA's
// issue time.
#pragma once
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace helm {

// The rare case of df_split (zero, tiny, huge, inf, NaN) by the converting instructions.
// Kept out of line: inlined, the compiler predicates it into every split, and its FP64
// instructions then occupy the FP64 pipe for every point (measured: the cycle-start pass
// at 85% of that pipe).
__device__ __noinline__ float2 df_split_rare(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

// x = hi + lo: hi takes the top 24 bits of x's significand and lo the next 23, on the
// integer pipes (re-biased exponents, the fraction bits moved by shifts, lo's integer
// scaled by a power of two).  Outside 2^-80 <= |x| < 2^128 (zero, tiny, huge, inf, NaN)
// the converting instructions round instead.
__device__ __forceinline__ float2 df_split(double x) {
  const unsigned xh = (unsigned)__double2hiint(x), xl = (unsigned)__double2loint(x);
  const unsigned e = (xh >> 20) & 0x7ffu;  // biased binary64 exponent
  if (e - 943u > 207u) return df_split_rare(x);
  const unsigned sign = xh & 0x80000000u;
  const unsigned t = (xh & 0x7fffffffu) - (896u << 20);  // exponent re-biased for binary32
  const float hi = __uint_as_float(sign | __funnelshift_l(xl, t, 3));
  // the 29 fraction bits below hi: their top 23 as the integer k (2^23 + k is exact in
  // binary32), worth k 2^(e - 1069)
  const float k = __fsub_rn(__uint_as_float(0x4b000000u | ((xl >> 6) & 0x7fffffu)), 8388608.0f);
  const float scale = __uint_as_float(sign | ((e - 942u) << 23));
  return make_float2(hi, __fmul_rn(k, scale));
}
__device__ __forceinline__ float4 df_split(double2 v) {
  const float2 a = df_split(v.x), b = df_split(v.y);
  return make_float4(a.x, a.y, b.x, b.y);
}

// a + b = t + r exactly (TwoSum)
__device__ __forceinline__ void df_two_sum(float a, float b, float& t, float& r) {
  t = __fadd_rn(a, b);
  const float z = __fsub_rn(t, a);
  r = __fadd_rn(__fsub_rn(a, __fsub_rn(t, z)), __fsub_rn(b, z));
}

// (s, c) += (ah + al)(bh + bl): s carries the running sum exactly updated by TwoSum, c
// the accumulated low-order parts (TwoProduct error, cross terms; al bl lies below the
// kept precision and is dropped).
__device__ __forceinline__ void df_mac(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, fmaf(al, bh, e));
  float t, r;
  df_two_sum(s, p, t, r);
  c = __fadd_rn(c, __fadd_rn(r, e));
  s = t;
}

// (s, c) += (ah + al) b for a binary32 b (exact when b is a complex64 component): the
// product ah b exactly by TwoProduct, al b rounded once.
__device__ __forceinline__ void df_mac1(float& s, float& c, float ah, float al, float b) {
  const float p = __fmul_rn(ah, b);
  const float e = fmaf(al, b, fmaf(ah, b, -p));
  float t, r;
  df_two_sum(s, p, t, r);
  c = __fadd_rn(c, __fadd_rn(r, e));
  s = t;
}

// Complex accumulator of double-float sums: re = sr + cr, im = si + ci.
struct DfAcc {
  float sr, cr, si, ci;
};
// a += k v for a double-float complex k = {re.hi, re.lo, im.hi, im.lo} and a complex64 v.
// A real k (zero imaginary part: stencil coefficients outside the absorbing layers)
// takes two multiply-adds instead of four; the skipped products are exact zeros, whose
// TwoSum leaves (s, c) unchanged (up to the sign of a zero sum).
__device__ __forceinline__ void df_cmac(DfAcc& a, float4 k, float2 v) {
  df_mac1(a.sr, a.cr, k.x, k.y, v.x);
  df_mac1(a.si, a.ci, k.x, k.y, v.y);
  if (k.z != 0.0f || k.w != 0.0f) {
    df_mac1(a.sr, a.cr, -k.z, -k.w, v.y);
    df_mac1(a.si, a.ci, k.z, k.w, v.x);
  }
}
// a = k v (the first term of a sum: the TwoSum against a zero accumulator is skipped)
__device__ __forceinline__ DfAcc df_cmul_first(float4 k, float2 v) {
  DfAcc a;
  a.sr = __fmul_rn(k.x, v.x);
  a.cr = fmaf(k.y, v.x, fmaf(k.x, v.x, -a.sr));
  a.si = __fmul_rn(k.x, v.y);
  a.ci = fmaf(k.y, v.y, fmaf(k.x, v.y, -a.si));
  if (k.z != 0.0f || k.w != 0.0f) {
    df_mac1(a.sr, a.cr, -k.z, -k.w, v.y);
    df_mac1(a.si, a.ci, k.z, k.w, v.x);
  }
  return a;
}
// (ah + al) + (bh + bl), renormalised
__device__ __forceinline__ float2 df_add(float ah, float al, float bh, float bl) {
  float s, r;
  df_two_sum(ah, bh, s, r);
  r = __fadd_rn(r, __fadd_rn(al, bl));
  const float t = __fadd_rn(s, r);
  return make_float2(t, __fsub_rn(r, __fsub_rn(t, s)));
}
__device__ __forceinline__ float4 df_cadd(float4 a, float4 b) {
  const float2 re = df_add(a.x, a.y, b.x, b.y), im = df_add(a.z, a.w, b.z, b.w);
  return make_float4(re.x, re.y, im.x, im.y);
}

// (s, c) renormalised so that c is below one unit in the last place of s (Fast2Sum;
// exact when |s| >= |c|, otherwise off by a rounding of the small c).  Done once per
// point, it keeps c from growing with the number of terms, so the rounding of the
// additions into c stays proportional to the sum's magnitude.
__device__ __forceinline__ void df_renorm(float& s, float& c) {
  const float t = __fadd_rn(s, c);
  c = __fsub_rn(c, __fsub_rn(t, s));
  s = t;
}

// The accumulated (s, c) as one binary64 value (widened on the integer pipes, one FP64 add).
__device__ __forceinline__ double df_value(float s, float c) { return widen(s) + widen(c); }

}  // namespace helm
