// Packed double-float arithmetic: two independent df64 accumulations per
// operation.
//
// sm_100-class GPUs execute the f32x2 forms of add, sub, mul and fma as one
// instruction that does both lanes (IEEE binary32, round to nearest, no
// flush to zero). The binary32 pipe still does 32 lane-operations per clock
// per scheduler, so a packed instruction takes the pipe for two cycles, but
// it takes one issue slot instead of two (measured on GB300: packed FMA at
// the scalar lane rate in half the warp instructions).
//
// Every function below performs, in each lane, exactly the operation
// sequence of its scalar counterpart in sem_df64.cuh (Dekker's product via
// FMA, Knuth's TwoSum, the compensated dot-product accumulator of Ogita, Rump
// & Oishi), so each lane's result is bit-identical to the scalar code on the
// same inputs. Negated operands are folded into the packed instructions by
// the compiler (measured: no extra instruction).
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

// two compensated accumulators: value s + c per lane
struct Acc {
  float2 s, c;
};

// s + e = a + b exactly (TwoSum)
__device__ __forceinline__ void two_sum(float2 a, float2 b, float2 &s, float2 &e) {
  s = add(a, b);
  const float2 v = sub(s, a);
  e = add(sub(a, sub(s, v)), sub(b, v));
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

}  // namespace dfx
