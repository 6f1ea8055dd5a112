// dfloat.cuh -- double-float helpers (a value held as an unevaluated sum h + l
// of two FP32 numbers) shared by the tensor-core contractions (k_oz.cu) and
// the double-float QR blocks (k_qr_df.cu).  The FP64 pipe of this GPU runs at
// about 1/62 of the FP32 rate, so FP64-accurate work that is not a dense
// contraction is cheaper in pairs of FP32 numbers, and conversions to FP64 are
// built with integer operations.
#pragma once
#include <stdint.h>

namespace htgb {
namespace {

// Error-free sums in FP32 (Knuth's two-sum, Dekker's fast two-sum for |a| >= |b|).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// (h + l) 2^E as an FP64 bit pattern, for |l| <= ulp(h) / 2: h's 24-bit
// significand at bit 52, l's added at its offset (bits below 2^-52 of h's
// scale cut), renormalised by one place if the sum crossed a power of two.
// Subnormal h, and results below the FP64 normal range, give zero; results
// above it, and h = Inf or NaN, give Inf of h's sign.
__device__ __forceinline__ unsigned long long df_to_f64_bits(float h, float l, int E) {
  const uint32_t bh = __float_as_uint(h);
  const int eh = (int)((bh >> 23) & 0xFFu);
  if (eh == 0) return 0ull;
  long long W = (long long)((bh & 0x7FFFFFu) | 0x800000u) << 29;  // [2^52, 2^53)
  const uint32_t bl = __float_as_uint(l);
  const int el = (int)((bl >> 23) & 0xFFu);
  if (el != 0) {
    const long long ml = (long long)((bl & 0x7FFFFFu) | 0x800000u);
    const int sh = el - eh + 29;  // <= 5
    const long long lp = sh >= 0 ? (ml << sh) : (sh > -40 ? (ml >> (-sh)) : 0ll);
    W = ((bl ^ bh) >> 31) ? W - lp : W + lp;
  }
  int ex = eh - 127 + 1023 + E;
  if (W >= (1ll << 53)) {
    W >>= 1;
    ++ex;
  } else if (W < (1ll << 52)) {
    W <<= 1;
    --ex;
  }
  if (ex <= 0) return 0ull;
  const unsigned long long sign = (unsigned long long)(bh >> 31) << 63;
  if (ex >= 2047 || eh == 255) return sign | 0x7FF0000000000000ull;
  return sign | ((unsigned long long)ex << 52) | ((unsigned long long)W & 0xFFFFFFFFFFFFFull);
}

// (p, e) with p + e = (ah + al)(bh + bl) up to the al bl term and the
// rounding of e (both below 2^-48 of the product).
__device__ __forceinline__ void df_prod(float ah, float al, float bh, float bl, float &p, float &e) {
  p = __fmul_rn(ah, bh);
  e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
}

// (h, l) = a + b for canonical pairs.
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float &h, float &l) {
  float s, t;
  two_sum(ah, bh, s, t);
  t = __fadd_rn(t, __fadd_rn(al, bl));
  fast_two_sum(s, t, h, l);
}

// (h, l) = a b.
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &h, float &l) {
  float p, e;
  df_prod(ah, al, bh, bl, p, e);
  fast_two_sum(p, e, h, l);
}

// x 2^-E as a pair (|x| < 2^E): h = x's sign, scaled exponent and top 23
// fraction bits; l = the next 23 fraction bits at their place.  Zero, FP64
// subnormals and results below 2^-126 give zero (l alone below 2^-126 is
// dropped).
__device__ __forceinline__ void df_from_f64(double x, int E, float &h, float &l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const int fe = ex - 1023 - E + 127;  // biased FP32 exponent of x 2^-E
  h = 0.0f;
  l = 0.0f;
  if (ex == 0 || fe < 1) return;
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  h = __uint_as_float(sign | ((uint32_t)fe << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu));
  const uint32_t k = (uint32_t)(b >> 6) & 0x7FFFFFu;  // fraction bits 28 .. 6
  if (k != 0u && fe > 46) {
    // k exactly as a float (1.5 2^23 trick without the half), times 2^(fe - 127 - 46)
    const float kf = __fsub_rn(__uint_as_float(0x4B000000u | k), 8388608.0f);
    l = __uint_as_float(__float_as_uint(__fmul_rn(kf, __uint_as_float((uint32_t)(fe - 46) << 23))) | sign);
  }
}

__device__ __forceinline__ double df_to_f64(float h, float l, int E) {
  return __longlong_as_double((long long)df_to_f64_bits(h, l, E));
}

}  // namespace
}  // namespace htgb
