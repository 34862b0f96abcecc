// Double-float ("df64") arithmetic on the binary32 pipe.
//
// A value is the unevaluated sum hi + lo of two binary32 numbers. Products
// are made exact with one FMA (Dekker's product via fused multiply-add),
// sums with Knuth's TwoSum, and dot products accumulate the high parts with
// TwoSum and every rounding error in a separate low accumulator (the
// compensated dot product of Ogita, Rump & Oishi 2005). All operations use
// the _rn intrinsics so the compiler cannot fuse or reorder them.
//
// Conversions between binary64 and df64 use integer bit manipulation only:
// on this GPU binary64<->binary32 conversion instructions run at the (very
// low) binary64 rate, while integer and binary32 instructions run at full
// rate.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace df {

__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }

// s + e = a + b exactly (TwoSum, 6 flops)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = add(a, b);
  const float v = sub(s, a);
  e = add(sub(a, sub(s, v)), sub(b, v));
}

// s + e = a + b exactly when |a| >= |b| (Fast2Sum, 3 flops)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = add(a, b);
  e = sub(b, sub(s, a));
}

// Compensated accumulator: value = s + c, c collects every rounding error.
struct Acc {
  float s, c;
};

// acc = (ah + al) * (bh + bl), first term (no addition error yet)
__device__ __forceinline__ Acc mul_first(float ah, float al, float bh, float bl) {
  Acc r;
  r.s = mul(ah, bh);
  float e = fmaf(ah, bh, -r.s);  // exact error of the product
  e = fmaf(ah, bl, e);
  r.c = fmaf(al, bh, e);
  return r;
}

// acc += (ah + al) * (bh + bl)
__device__ __forceinline__ void mac(Acc &acc, float ah, float al, float bh, float bl) {
  const float p = mul(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  float t, err;
  two_sum(acc.s, p, t, err);
  acc.s = t;
  acc.c = add(acc.c, add(err, e));
}

// acc += (bh + bl) for a df value b
__device__ __forceinline__ void acc_add(Acc &acc, float bh, float bl) {
  float t, err;
  two_sum(acc.s, bh, t, err);
  acc.s = t;
  acc.c = add(acc.c, add(err, bl));
}

// normalised (hi, lo) of an accumulator: TwoSum, valid for any magnitudes
__device__ __forceinline__ float2 norm(const Acc &a) {
  float h, l;
  two_sum(a.s, a.c, h, l);
  return make_float2(h, l);
}

// binary64 -> (hi, lo): hi = the leading 24 bits of x (truncated), lo = the
// next 29 bits rounded to binary32, so hi + lo = x to ~2^-48 relative.
// |x| < 2^-126 becomes 0 (signed); infinities and NaN keep their class.
__device__ __forceinline__ float2 from_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
  const int e = (int)((bh >> 20) & 0x7FFu);
  const unsigned sgn = bh & 0x80000000u;
  const unsigned mh = ((bh & 0xFFFFFu) << 3) | (bl >> 29);
  const int ef = e - 896;  // binary32 biased exponent
  if (ef <= 0) return make_float2(__uint_as_float(sgn), 0.0f);
  if (ef >= 255) {
    const unsigned nan = ((bh & 0xFFFFFu) | bl) ? 0x400000u : 0u;
    return make_float2(__uint_as_float(sgn | 0x7F800000u | nan), 0.0f);
  }
  const float hi = __uint_as_float(sgn | ((unsigned)ef << 23) | mh);
  const float scale = __uint_as_float((unsigned)ef << 23);  // 2^(e - 1023)
  float lo = mul(mul(__uint2float_rn(bl & 0x1FFFFFFFu), 0x1p-52f), scale);
  lo = __uint_as_float(__float_as_uint(lo) ^ sgn);
  return make_float2(hi, lo);
}

// normalised (hi, lo) -> nearest binary64 (|lo| <= ulp(hi)/2 assumed):
// the binary64 bits of hi plus lo counted in binary64 ulps of hi, added as
// an integer (carries across a binade are handled by the IEEE ordering).
__device__ __forceinline__ double to_f64(float h, float l) {
  const unsigned hb = __float_as_uint(h);
  const unsigned ef = (hb >> 23) & 0xFFu;
  const unsigned sgn = hb & 0x80000000u;
  const unsigned m = hb & 0x7FFFFFu;
  // the binary64 bits of hi (exact)
  long long D = (long long)(((unsigned long long)(sgn | ((ef + 896u) << 20) | (m >> 3)) << 32) |
                            ((unsigned long long)(m & 7u) << 29));
  if (ef < 54u || ef == 255u) {  // rare: integer bit work only, no binary64 arithmetic
    if (ef == 255u) return __longlong_as_double((long long)((unsigned long long)(sgn | 0x7FF00000u | (m ? 0x80000u : 0u)) << 32));
    if (ef == 0u) return __longlong_as_double((long long)((unsigned long long)sgn << 32));  // zero (binary32 subnormals too)
    return __longlong_as_double(D);  // |hi| < 2^-73: hi alone (|lo| < 2^-24 |hi|)
  }
  // lo in ulps of hi (2^(E-52), E = ef - 127): scale 2^(179 - ef); when hi is
  // a power of two and lo points toward zero the sum lies in the binade
  // below, whose ulp is half as large: scale by 2^(180 - ef)
  const bool down = (m == 0u) && (l != 0.0f) && (((__float_as_uint(l) ^ hb) & 0x80000000u) != 0u);
  const unsigned sexp = (down ? 307u : 306u) - ef;
  const float kf = mul(l, __uint_as_float(sexp << 23));
  const long long k = (long long)__float2int_rn(kf);
  D += sgn ? -k : k;
  return __longlong_as_double(D);
}

// Biased binary64 exponent of x (0 for zero and subnormals), or 0 for
// infinities and NaN so that they do not set an element's scale.
__device__ __forceinline__ int exp_field(double x) {
  const int e = (int)((((unsigned long long)__double_as_longlong(x)) >> 52) & 0x7FFull);
  return e == 0x7FF ? 0 : e;
}

// Power-of-two scaling for values outside the binary32 exponent range: an
// element's values are carried as x 2^-sh with sh the unbiased exponent of
// its largest |x|, so the largest maps to [1, 2) and everything below it by
// up to 2^-126 stays representable (smaller values flush to zero, below the
// accuracy the operator promises relative to the element's largest value).
// sh comes from exp_field: sh = emax - 1023.
//
// (hi, lo) of x 2^-sh; infinities and NaN keep their class. The binary32
// exponent of the scaled value is computed once from the binary64 exponent
// field; the common path is the bit work of from_f64.
__device__ __forceinline__ float2 from_f64_scaled(double x, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
  const int e = (int)((bh >> 20) & 0x7FFu);
  const unsigned sgn = bh & 0x80000000u;
  const int ef = e - 896 - sh;  // binary32 biased exponent of x 2^-sh
  if (e == 0x7FF || e == 0 || ef <= 0 || ef >= 255) {  // rare: not finite, zero, or out of range once scaled
    if (e == 0x7FF) return from_f64(x);
    if (e == 0 || ef <= 0) return make_float2(__uint_as_float(sgn), 0.0f);
    return make_float2(__uint_as_float(sgn | 0x7F800000u), 0.0f);
  }
  const unsigned mh = ((bh & 0xFFFFFu) << 3) | (bl >> 29);
  const float hi = __uint_as_float(sgn | ((unsigned)ef << 23) | mh);
  const float scale = __uint_as_float((unsigned)ef << 23);  // 2^(unbiased exponent of hi)
  float lo = mul(mul(__uint2float_rn(bl & 0x1FFFFFFFu), 0x1p-52f), scale);
  lo = __uint_as_float(__float_as_uint(lo) ^ sgn);
  return make_float2(hi, lo);
}

// nearest binary64 of (h + l) 2^sh (the inverse scaling of from_f64_scaled):
// to_f64 with the exponent of the result raised by sh
__device__ __forceinline__ double to_f64_scaled(float h, float l, int sh) {
  const unsigned hb = __float_as_uint(h);
  const unsigned ef = (hb >> 23) & 0xFFu;
  const int e64 = (int)ef + 896 + sh;  // binary64 biased exponent of hi 2^sh
  if (ef < 54u || ef == 255u || e64 < 2 || e64 > 0x7FE) {  // rare: tiny, zero, not finite, or out of range
    const double d = to_f64(h, l);
    if (sh == 0) return d;
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7FFull);
    if (e == 0 || e == 0x7FF) return d;
    const int es = e + sh;
    if (es >= 1 && es <= 0x7FE) return __longlong_as_double((long long)(b + ((unsigned long long)(long long)sh << 52)));
    const unsigned long long sg = b & 0x8000000000000000ull;  // flushed to a signed zero, or infinity
    return __longlong_as_double((long long)(es < 1 ? sg : (sg | 0x7FF0000000000000ull)));
  }
  const unsigned sgn = hb & 0x80000000u;
  const unsigned m = hb & 0x7FFFFFu;
  long long D = (long long)(((unsigned long long)(sgn | ((unsigned)e64 << 20) | (m >> 3)) << 32) |
                            ((unsigned long long)(m & 7u) << 29));
  // lo in binary64 ulps of hi (as in to_f64; independent of the scaling)
  const bool down = (m == 0u) && (l != 0.0f) && (((__float_as_uint(l) ^ hb) & 0x80000000u) != 0u);
  const unsigned sexp = (down ? 307u : 306u) - ef;
  const float kf = mul(l, __uint_as_float(sexp << 23));
  const long long k = (long long)__float2int_rn(kf);
  D += sgn ? -k : k;
  return __longlong_as_double(D);
}

}  // namespace df
