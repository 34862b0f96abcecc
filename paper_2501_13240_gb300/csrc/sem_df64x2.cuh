// Packed double-float arithmetic: two independent df64 values per operation.
//
// sm_100-class GPUs execute the f32x2 forms of add, sub, mul and fma as one
// instruction that does both lanes (IEEE binary32, round to nearest, no
// flush to zero). The binary32 pipe still does 32 lane-operations per clock
// per scheduler, so a packed instruction takes the pipe for two cycles, but
// it takes one issue slot instead of two: an issue-bound kernel built from
// these frees half of its arithmetic issue slots for loads, integer and
// conversion work.
//
// Every function below performs, in each lane, exactly the operation
// sequence of its scalar counterpart in sem_df64.cuh (Dekker's product via
// FMA, Knuth's TwoSum, Fast2Sum, the compensated dot-product accumulator of
// Ogita, Rump & Oishi), so each lane's result is bit-identical to the scalar
// code on the same inputs. Negated operands are folded into the packed
// instructions by the compiler.
#pragma once

#include <cuda_runtime.h>

namespace dfx {

__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// two double-float values: lane 0 = (h.x, l.x), lane 1 = (h.y, l.y)
struct V {
  float2 h, l;
};

// two compensated accumulators: value s + c per lane
struct Acc {
  float2 s, c;
};

__device__ __forceinline__ V make_v(float2 a, float2 b) {  // lane 0 from a = (hi, lo), lane 1 from b
  V r;
  r.h = make_float2(a.x, b.x);
  r.l = make_float2(a.y, b.y);
  return r;
}

// s + e = a + b exactly (TwoSum)
__device__ __forceinline__ void two_sum(float2 a, float2 b, float2 &s, float2 &e) {
  s = add(a, b);
  const float2 v = sub(s, a);
  e = add(sub(a, sub(s, v)), sub(b, v));
}

// s + e = a - b exactly: TwoSum(a, -b) with the negation taken by the
// subtractions (same bits as the scalar TwoSum of a and -b)
__device__ __forceinline__ void two_diff(float2 a, float2 b, float2 &s, float2 &e) {
  s = sub(a, b);
  const float2 v = sub(s, a);
  e = sub(sub(a, sub(s, v)), add(b, v));
}

// s + e = a + b exactly when |a| >= |b| (Fast2Sum)
__device__ __forceinline__ void fast_two_sum(float2 a, float2 b, float2 &s, float2 &e) {
  s = add(a, b);
  e = sub(b, sub(s, a));
}

// acc = (ah + al) * (bh + bl)
__device__ __forceinline__ Acc mul_first(float2 ah, float2 al, float2 bh, float2 bl) {
  Acc r;
  r.s = mul(ah, bh);
  float2 e = fma(ah, bh, neg(r.s));
  e = fma(ah, bl, e);
  r.c = fma(al, bh, e);
  return r;
}

// acc += (ah + al) * (bh + bl)
__device__ __forceinline__ void mac(Acc &acc, float2 ah, float2 al, float2 bh, float2 bl) {
  const float2 p = mul(ah, bh);
  float2 e = fma(ah, bh, neg(p));
  e = fma(ah, bl, e);
  e = fma(al, bh, e);
  float2 t, err;
  two_sum(acc.s, p, t, err);
  acc.s = t;
  acc.c = add(acc.c, add(err, e));
}

// acc += (bh + bl)
__device__ __forceinline__ void acc_add(Acc &acc, float2 bh, float2 bl) {
  float2 t, err;
  two_sum(acc.s, bh, t, err);
  acc.s = t;
  acc.c = add(acc.c, add(err, bl));
}

// normalised (hi, lo) of an accumulator (TwoSum: any magnitudes)
__device__ __forceinline__ V norm(const Acc &a) {
  V r;
  two_sum(a.s, a.c, r.h, r.l);
  return r;
}

// normalised (hi, lo) when |s| >= |c| (Fast2Sum)
__device__ __forceinline__ V fast_norm(const Acc &a) {
  V r;
  fast_two_sum(a.s, a.c, r.h, r.l);
  return r;
}

}  // namespace dfx
