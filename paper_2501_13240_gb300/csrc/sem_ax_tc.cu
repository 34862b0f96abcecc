// binary64-accurate Helmholtz operator at N = 7 with the 1-D contractions on
// the tensor pipe (Sec. 2.2: the leading-order work is dense (p+1)x(p+1)
// tensor contractions shared by all elements).
//
// Why: the double-float operator (sem_ax_df64.cu) spends three quarters of
// its binary32 lane operations in the six 1-D contractions (about 59 per
// point and contraction: every multiply-add is an error-free product plus a
// compensated sum). Here each contraction is an exact integer computation on
// fp16 tensor cores (mma.sync m16n8k16, f32 accumulate), in the manner of
// the Ozaki scheme (Ozaki, Ogita, Oishi & Rump 2012): both operands are cut
// into digits on a common fixed-point grid, every digit product is exact,
// and digit products of equal weight are summed exactly in binary32.
//
// Digits. A value y with |y| < 1 is written y = sum_j d_j 2^-10(j+1),
// j = 0..4, with integer digits (|d_0| <= 1024, |d_j| <= 576 otherwise,
// each exact in fp16); the truncation error is below 2^-50. D is sliced the
// same way as D/32 (|D| <= 18.94 at N = 7), once on the host. The digit
// products of level L = i + j (i, j <= 4) have weight 2^-10(L+2); the 15
// products of levels 0..4 are kept, the rest is below 2^-47 of |D||y|.
// Every level sum is an integer below 2^23.4 (bound computed from D's
// digits, for up to two contraction directions summed), so the f32
// accumulation inside the tensor core is exact whatever its order.
// Recombining the five levels into a double-float costs 16 binary32
// operations (integer part of level 1 added to level 0 exactly, its fraction
// and level 2 summed exactly, levels 3 and 4 below 2^-32 of the result).
//
// Scales. An element's input u is carried as x = u 2^-su with |x| < 1 (su
// from the largest binary64 exponent of the element, so any finite input
// works); the metric outputs v are digit-sliced at a second power-of-two
// scale 2^-sv of the element's largest |v|.
//
// Threads: one element per 128-thread CTA, four warps. In P0, P2 and P4
// warp w owns the planes t = 2w, 2w + 1 and lane (g, q) the point pair
// r = 2q, 2q + 1 at s = g of each; the digits of a point pair are one f16x2
// word. The digits go to shared memory, and each contraction pass works on
// 24 line groups (three directions x eight planes or rows, six per warp):
// D's digits are the A operand, held in two fixed register quads so that
// each accumulator collects digit products of one level, and the group's
// digits are the B operand, loaded by ldmatrix (.trans where the lines run
// across the shared-memory rows). Each group's five levels are recombined
// to double-float and stored to the direction's shared tile.
//
// Phases per element:
//   P0 gather u, element scale su, digits of x (registers and shared memory)
//   P1 forward contractions (six mma per line group) and recombination to
//      double-float: ur, us, ut in the shared tiles
//   P2 metric (wr, ws, wt) = G (ur, us, ut) in double-float; element scale
//      sv of the result; digits of the three fields to shared memory
//   P3 transposed contractions of the three fields into the shared tiles
//   P4 sum, Helmholtz term, scale back to binary64, scatter (atomics or the
//      deterministic E-vector), p.w partial
#include <math.h>

#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "sem_df64.cuh"
#include "sem_df64x2.cuh"
#include "sem_internal.h"

namespace {

constexpr int NP = 8, N3 = 512;
constexpr int NSL = 5;             // digit slices per operand
constexpr double kDScale = 32.0;   // D is sliced as D / 32
constexpr int kMinBlocks = 5;      // resident 128-thread CTAs per SM the register budget aims at

// D's digits as mma fragment registers, per lane: [0][j][lane] = (D_j[g][2q],
// D_j[g][2q+1]) (forward: B of the r-contraction, A of s and t),
// [1][j][lane] = (D_j[2q][g], D_j[2q+1][g]) (the transposed contractions)
__device__ uint32_t g_dig[2][NSL][32];

// The even-odd split of D for the register-resident kernel's t-lines, whose
// two columns are the lanes of packed instructions: entry [tr][0][i 4 + m] =
// A (i, m) = (M(i, m) + M(i, 7 - m)) / 2 and [tr][1][...] = Bq = (M(i, m) -
// M(i, 7 - m)) / 2, M = D (tr 0) or D^T (tr 1), each as (hi, hi, lo, lo) so
// that one 16-byte load gives both lanes' operands.
__constant__ float4 c_tq[2][2][16];

std::mutex g_dig_mu;
unsigned g_dig_ready = 0;  // bit per device

uint16_t f16_bits_of_int(int v) {
  // exact fp16 encoding of an integer with |v| <= 2048
  if (v == 0) return 0;
  const uint16_t sgn = v < 0 ? 0x8000u : 0u;
  int a = v < 0 ? -v : v;
  int e = 0;
  while ((a >> e) > 1) ++e;            // 2^e <= a < 2^(e+1)
  const int mant = (a << (10 - e)) & 0x3FF;  // 10 stored bits (exact: a has <= 11 significant bits)
  return (uint16_t)(sgn | ((e + 15) << 10) | mant);
}

int ensure_digits(int device) {
  std::lock_guard<std::mutex> lk(g_dig_mu);
  if (device < 32 && (g_dig_ready >> device) & 1u) return SEM_OK;
  double xi[SEM_MAXNP], rho[SEM_MAXNP], D[SEM_MAXNP * SEM_MAXNP];
  if (int rc = sem_gll_host(NP - 1, xi, rho, D)) return rc;
  // digits of D/32: d = round(y 1024), y <- y 1024 - d (exact in binary64)
  int dig[NSL][NP][NP];
  for (int i = 0; i < NP; ++i)
    for (int m = 0; m < NP; ++m) {
      double y = D[i * NP + m] / kDScale;
      if (!(fabs(y) < 1.0)) return sem_fail(SEM_ERR_INVALID_ARG, "tensor-core operator: D out of range");
      for (int j = 0; j < NSL; ++j) {
        y *= 1024.0;
        const double d = nearbyint(y);
        dig[j][i][m] = (int)d;
        y -= d;
      }
    }
  std::vector<uint32_t> tab(2 * NSL * 32);
  for (int j = 0; j < NSL; ++j)
    for (int lane = 0; lane < 32; ++lane) {
      const int g = lane >> 2, q = lane & 3;
      tab[(0 * NSL + j) * 32 + lane] = (uint32_t)f16_bits_of_int(dig[j][g][2 * q]) |
                                       ((uint32_t)f16_bits_of_int(dig[j][g][2 * q + 1]) << 16);
      tab[(1 * NSL + j) * 32 + lane] = (uint32_t)f16_bits_of_int(dig[j][2 * q][g]) |
                                       ((uint32_t)f16_bits_of_int(dig[j][2 * q + 1][g]) << 16);
    }
  SEM_CUDA(cudaMemcpyToSymbol(g_dig, tab.data(), sizeof(uint32_t) * tab.size()));
  std::vector<float4> tq(2 * 2 * 16);
  for (int tr = 0; tr < 2; ++tr) {
    auto M = [&](int i, int m) { return tr ? D[m * NP + i] : D[i * NP + m]; };
    for (int i = 0; i < 4; ++i)
      for (int m = 0; m < 4; ++m)
        for (int ab = 0; ab < 2; ++ab) {
          const double v = 0.5 * (M(i, m) + (ab ? -1.0 : 1.0) * M(i, NP - 1 - m));
          const float hi = (float)v, lo = (float)(v - (double)hi);
          tq[(tr * 2 + ab) * 16 + i * 4 + m] = make_float4(hi, hi, lo, lo);
        }
  }
  SEM_CUDA(cudaMemcpyToSymbol(c_tq, tq.data(), sizeof(float4) * tq.size()));
  if (device < 32) g_dig_ready |= 1u << device;
  return SEM_OK;
}

// ---------------------------------------------------------------- tensor-core primitives
// d = A B + c, m16n8k16, fp16 inputs, f32 accumulate
__device__ __forceinline__ void mma16(float &d0, float &d1, float &d2, float &d3, uint32_t a0, uint32_t a1,
                                      uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1, float c0, float c1,
                                      float c2, float c3) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%10,%11,%12,%13};"
      : "=f"(d0), "=f"(d1), "=f"(d2), "=f"(d3)
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(c0), "f"(c1), "f"(c2), "f"(c3));
}




__device__ __forceinline__ uint32_t pack_f16(float2 v) {
  const __half2 h = __floats2half2_rn(v.x, v.y);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// ---------------------------------------------------------------- packed binary32 pairs
// A thread's two points (r = 2q, 2q+1) are the two lanes of f32x2
// instructions: one issue slot for both (each lane does the scalar
// operation sequence).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return dfx::sub(a, b); }
__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }

// Digits of the pair y = (h + l) s1 2^-10 (|y| <= 1): s1 = 2^10 2^-scale,
// c2 = s1 2^10; out[j] = the fp16 pair of digit j. Round to nearest integer
// by the 1.5 2^23 shift. The low word enters at the third digit through an
// exact Fast2Sum (|r| >= |l c2| unless r = 0: there r is a multiple of
// ulp(h), and |l| < ulp(h)).
__device__ __forceinline__ void digits5(float2 h, float2 l, float s1, float c2, uint32_t (&out)[NSL]) {
  const float2 M = dup(12582912.0f), K = dup(1024.0f), S = dup(s1), C = dup(c2);
  float2 t = fma2(h, S, M);
  float2 d = sub2(t, M);
  out[0] = pack_f16(d);
  float2 r = fma2(h, S, neg2(d));
  t = fma2(r, K, M);
  d = sub2(t, M);
  out[1] = pack_f16(d);
  r = fma2(r, K, neg2(d));
  const float2 sm = fma2(l, C, r);
  const float2 z = sub2(sm, r);
  const float2 eps = fma2(l, C, neg2(z));
  t = fma2(sm, K, M);
  d = sub2(t, M);
  out[2] = pack_f16(d);
  r = fma2(sm, K, neg2(d));
  r = fma2(eps, K, r);
  t = fma2(r, K, M);
  d = sub2(t, M);
  out[3] = pack_f16(d);
  r = fma2(r, K, neg2(d));
  out[4] = pack_f16(mul2(r, K));  // rounded to 11 bits by the fp16 conversion
}

// The five level sums L_0..L_4 (exact integers) of an output pair, weight
// 2^-10(L+2) times sc, to normalised double-floats: (hi pair, lo pair).
__device__ __forceinline__ void recombine(float2 L0, float2 L1, float2 L2, float2 L3, float2 L4, float sc,
                                          float2 &H, float2 &Lo) {
  const float2 M = dup(12582912.0f);
  const float2 v1 = mul2(L1, dup(0x1p-10f));
  const float2 hi1 = sub2(add2(v1, M), M);  // integer part of level 1 (|v1| < 2^22)
  const float2 fr1 = sub2(v1, hi1);         // its fraction, exact
  const float2 A = add2(L0, hi1);           // integer below 2^24: exact
  const float2 B = fma2(L2, dup(0x1p-20f), fr1);  // on the 2^-20 grid, below 2^3: exact
  const float2 C = fma2(L4, dup(0x1p-10f), L3);   // levels 3, 4 in level-3 units (error < 2^-32)
  const float2 h = add2(A, B);              // Fast2Sum: exact when |A| >= 8, else A + B is exact
  const float2 e = sub2(B, sub2(h, A));
  const float2 l = fma2(C, dup(0x1p-30f), e);
  const float2 S = add2(h, l);
  const float2 T = sub2(l, sub2(S, h));
  H = mul2(S, dup(sc));
  Lo = mul2(T, dup(sc));
}

// ---------------------------------------------------------------- one 1-D contraction group
// D (or D^T) digits as the A operand in two fixed register quads:
//   QA = (D0 | D1 over k; D2 | D3 over k)  rows 0..7 / 8..15 = levels i, i + 2
//   QB = (D0 | D4;        D2 | 0)
// and the digits of 8 lines as B from shared memory, in three quads loaded
// by ldmatrix straight into the registers the MMAs read:
//   E = (u1, u0, u3, u2), O = (u2, u1, u4, u3), Zq = (u0, 0, 0, u0)
// Six MMAs, each into its own accumulator quad (no operand is ever moved):
//   QA x (u1;u0) -> (L1 | L3)   QA x (u2;u1) -> (L2 | L4)   QA x (u3;u2) -> (L3 | -)
//   QA x (u4;u3) -> (L4 | -)    QB x (u0;0)  -> (L0 | L2)   QB x (0;u0)  -> (L4 | -)
// ("-": products of levels 5, 6, not used). The level pairs are summed with
// exact binary32 additions (every partial sum is part of a level sum below
// 2^23.4). Returns the output pair (output index g, lines 2q, 2q+1).
__device__ __forceinline__ void contract(const uint4 &QA, const uint4 &QB, const uint4 &E, const uint4 &O,
                                         const uint4 &Zq, float sc, float2 &H, float2 &Lo) {
  float4 q1, q2, q3, q4, q5, q6;
  mma16(q1.x, q1.y, q1.z, q1.w, QA.x, QA.y, QA.z, QA.w, E.x, E.y, 0.f, 0.f, 0.f, 0.f);
  mma16(q2.x, q2.y, q2.z, q2.w, QA.x, QA.y, QA.z, QA.w, O.x, O.y, 0.f, 0.f, 0.f, 0.f);
  mma16(q3.x, q3.y, q3.z, q3.w, QA.x, QA.y, QA.z, QA.w, E.z, E.w, 0.f, 0.f, 0.f, 0.f);
  mma16(q4.x, q4.y, q4.z, q4.w, QA.x, QA.y, QA.z, QA.w, O.z, O.w, 0.f, 0.f, 0.f, 0.f);
  mma16(q5.x, q5.y, q5.z, q5.w, QB.x, QB.y, QB.z, QB.w, Zq.x, Zq.y, 0.f, 0.f, 0.f, 0.f);
  mma16(q6.x, q6.y, q6.z, q6.w, QB.x, QB.y, QB.z, QB.w, Zq.z, Zq.w, 0.f, 0.f, 0.f, 0.f);
  const float2 L0 = make_float2(q5.x, q5.y), L1 = make_float2(q1.x, q1.y);
  const float2 L2 = add2(make_float2(q2.x, q2.y), make_float2(q5.z, q5.w));
  const float2 L3 = add2(make_float2(q1.z, q1.w), make_float2(q3.x, q3.y));
  const float2 L4 = add2(add2(make_float2(q2.z, q2.w), make_float2(q4.x, q4.y)), make_float2(q6.x, q6.y));
  recombine(L0, L1, L2, L3, L4, sc, H, Lo);
}

// shared-memory digit planes of one field: slice j, plane t, row s holds the
// 8 r-values (16 bytes) at chunk (j 8 + t) 8 + (s ^ t) (the xor spreads the
// rows of every matrix an ldmatrix reads over all bank groups)
__device__ __forceinline__ int dig_word(int j, int t, int s, int q) { return (((j * 8 + t) * 8 + (s ^ t)) << 2) + q; }
constexpr int kDigWords = NSL * 256;  // one field's digit planes (5 KB)

__device__ __forceinline__ void ldsm4(uint32_t addr, uint4 &r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ void ldsm4t(uint32_t addr, uint4 &r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "r"(addr)
               : "memory");
}

// B quads of one group. DIR 0 (r): lines s, k = r at plane c (plain
// ldmatrix: the stored rows are the lines); DIR 1 (s): k = s, lines r at
// plane c (transposed); DIR 2 (t): k = t, lines r at row s = c (transposed).
// Lane L gives the address of row L & 7 of matrix L >> 3; the slices of the
// four matrices are (1, 0, 3, 2), (2, 1, 4, 3), (0, Z, Z, 0) for E, O, Zq.
struct LaneRows {
  uint32_t je, jo, j0;  // byte offsets of this lane's matrix slices in a field's digit planes
  bool zmat;            // this lane's Zq matrix is the zero matrix
  int row;
};

__device__ __forceinline__ LaneRows lane_rows(int lane) {
  LaneRows L;
  const int mat = lane >> 3;
  L.row = lane & 7;
  L.je = 1024u * (uint32_t)(mat ^ 1);                    // slices 1, 0, 3, 2
  L.jo = 1024u * (uint32_t)((mat & 1) ? mat : mat + 2);  // slices 2, 1, 4, 3
  L.j0 = 0u;
  L.zmat = (mat == 1 || mat == 2);
  return L;
}

template <int DIR>
__device__ __forceinline__ void load_group(uint32_t dig, uint32_t zrow, const LaneRows &L, int c, uint4 &E, uint4 &O,
                                           uint4 &Zq) {
  // row address of (plane t, row s): chunk (j 8 + t) 8 + (s ^ t), 16 bytes each
  const int t = DIR == 2 ? L.row : c, s = DIR == 2 ? c : L.row;
  const uint32_t rowoff = dig + 128u * (uint32_t)t + 16u * (uint32_t)(s ^ t);
  const uint32_t az = L.zmat ? zrow : rowoff + L.j0;
  if (DIR == 0) {
    ldsm4(rowoff + L.je, E);
    ldsm4(rowoff + L.jo, O);
    ldsm4(az, Zq);
  } else {
    ldsm4t(rowoff + L.je, E);
    ldsm4t(rowoff + L.jo, O);
    ldsm4t(az, Zq);
  }
}

__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// one output pair of the metric step, g0 u0 + g1 u1 + g2 u2, in double-float
// (hi pair, lo pair) for the two points
__device__ __forceinline__ void metric_row2(const float2 (&gh)[6], const float2 (&gl)[6], int i0, int i1, int i2,
                                            const float2 (&uh)[3], const float2 (&ul)[3], float2 &oh, float2 &ol) {
  dfx::Acc a = dfx::mul_first(gh[i0], gl[i0], uh[0], ul[0]);
  dfx::mac(a, gh[i1], gl[i1], uh[1], ul[1]);
  dfx::mac(a, gh[i2], gl[i2], uh[2], ul[2]);
  oh = add2(a.s, a.c);  // Fast2Sum (|s| >= |c|)
  ol = sub2(a.c, sub2(oh, a.s));
}

__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((unsigned)(k + 127) << 23); }

// biased binary32 exponent of the larger of a pair (NaN/inf excluded)
__device__ __forceinline__ int fexp2(float2 h) {
  const unsigned a = __float_as_uint(h.x) & 0x7F800000u, b = __float_as_uint(h.y) & 0x7F800000u;
  const unsigned m = max(a == 0x7F800000u ? 0u : a, b == 0x7F800000u ? 0u : b);
  return (int)(m >> 23);
}

// the two inputs of a point pair: gathered through the map (assembled), or
// from the caller's E-vector (only 8-byte alignment is promised there)
template <bool ASSEMBLED>
__device__ __forceinline__ void load_u(const double *__restrict__ u, int2 gi, int64_t l, double (&v)[2]) {
  if (ASSEMBLED) {
    v[0] = gi.x >= 0 ? u[gi.x] : 0.0;
    v[1] = gi.y >= 0 ? u[gi.y] : 0.0;
  } else {
    v[0] = u[l];
    v[1] = u[l + 1];
  }
}

// double-float values in shared memory: a point pair (p even, p + 1) is
// (h_p, h_p+1, l_p, l_p+1); single points are written into their slots
__device__ __forceinline__ void st_pair(float2 *base, int p, float2 h, float2 l) {
  *reinterpret_cast<float4 *>(base + p) = make_float4(h.x, h.y, l.x, l.y);
}
__device__ __forceinline__ void ld_pair(const float2 *base, int p, float2 &h, float2 &l) {
  const float4 v = *reinterpret_cast<const float4 *>(base + p);
  h = make_float2(v.x, v.y);
  l = make_float2(v.z, v.w);
}
__device__ __forceinline__ void st_one(float2 *base, int p, float h, float l) {
  float *f = reinterpret_cast<float *>(base + (p & ~1));
  f[p & 1] = h;
  f[2 + (p & 1)] = l;
}

// Groups [c0, c1) of one direction, one per iteration (the four warps of
// an element give the overlap). The outputs go to the direction's tile: r as
// single points (its pair runs along s), s and t as point pairs along r.
template <int DIR>
__device__ __forceinline__ void contract_dir(uint32_t dig, uint32_t zrow, const LaneRows &L, int c0, int c1,
                                             const uint4 &QA, const uint4 &QB, float sc, int lane, float2 *o) {
  const int g = lane >> 2, q = lane & 3;
#pragma unroll 1
  for (int c = c0; c < c1; ++c) {
    uint4 E, O, Zq;
    load_group<DIR>(dig, zrow, L, c, E, O, Zq);
    float2 H, Lo;
    contract(QA, QB, E, O, Zq, sc, H, Lo);
    if (DIR == 0) {  // (r_out = g, s = 2q, 2q + 1) at plane c
      const int p = g + 16 * q + 64 * c;
      st_one(o, p, H.x, Lo.x);
      st_one(o, p + 8, H.y, Lo.y);
    } else if (DIR == 1) {  // (s_out = g, r = 2q, 2q + 1) at plane c
      st_pair(o, 2 * q + 8 * g + 64 * c, H, Lo);
    } else {  // (t_out = g, r = 2q, 2q + 1) at row s = c
      st_pair(o, 2 * q + 8 * c + 64 * g, H, Lo);
    }
  }
}

// The 24 line groups of one pass (3 directions x 8), 6 per warp:
// warp 0: r 0..5 | warp 1: r 6..7, s 0..3 | warp 2: s 4..7, t 0..1 | warp 3: t 2..7.
// per_dir: the transposed pass, whose three fields have their own digit
// planes (kDigWords apart).
__device__ __forceinline__ void contract_pass(uint32_t dig0, uint32_t zrow, bool per_dir, const uint4 &QA,
                                              const uint4 &QB, float sc, int wp, int lane, float2 *oR, float2 *oS,
                                              float2 *oT) {
  const LaneRows L = lane_rows(lane);
  const uint32_t fs = per_dir ? 4u * kDigWords : 0u;
  switch (wp) {
    case 0:
      contract_dir<0>(dig0, zrow, L, 0, 6, QA, QB, sc, lane, oR);
      break;
    case 1:
      contract_dir<0>(dig0, zrow, L, 6, 8, QA, QB, sc, lane, oR);
      contract_dir<1>(dig0 + fs, zrow, L, 0, 4, QA, QB, sc, lane, oS);
      break;
    case 2:
      contract_dir<1>(dig0 + fs, zrow, L, 4, 8, QA, QB, sc, lane, oS);
      contract_dir<2>(dig0 + 2 * fs, zrow, L, 0, 2, QA, QB, sc, lane, oT);
      break;
    default:
      contract_dir<2>(dig0 + 2 * fs, zrow, L, 2, 8, QA, QB, sc, lane, oT);
      break;
  }
}

// Threads: one element per 128-thread CTA, four warps; warp w owns planes
// t = 2w, 2w + 1, lane (g, q) the point pair r = 2q, 2q + 1 at s = g of each.
constexpr int kThreads = 128;

template <bool ASSEMBLED, bool HELM>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_ax_tc(int64_t E, const float2 *__restrict__ Gdf, const float2 *__restrict__ Bdf, float2 h1, float2 h2,
            const double *__restrict__ u, double *__restrict__ w, const int32_t *__restrict__ l2gm,
            double *__restrict__ pw_partial, double *__restrict__ wloc, const int *__restrict__ skip,
            const int32_t *__restrict__ elist) {
  if (skip != nullptr && *skip != 0) return;
  __shared__ __align__(16) float2 sR[N3];
  __shared__ __align__(16) float2 sS[N3];
  __shared__ __align__(16) float2 sT[N3];
  __shared__ __align__(16) uint32_t sDig[3 * kDigWords];  // digits of u, then of (wr, ws, wt)
  __shared__ __align__(16) uint32_t sZero[32];             // an 8x8 zero matrix for ldmatrix
  __shared__ int s_red[8];
  __shared__ double s_pw[4];
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31, g = lane >> 2, q = lane & 3;
  if (tid < 32) sZero[tid] = 0u;
  // D's digits as the two A quads, forward (D) and transposed (D^T)
  const uint4 FA = make_uint4(g_dig[0][0][lane], g_dig[0][2][lane], g_dig[0][1][lane], g_dig[0][3][lane]);
  const uint4 FB = make_uint4(g_dig[0][0][lane], g_dig[0][2][lane], g_dig[0][4][lane], 0u);
  const uint4 TA = make_uint4(g_dig[1][0][lane], g_dig[1][2][lane], g_dig[1][1][lane], g_dig[1][3][lane]);
  const uint4 TB = make_uint4(g_dig[1][0][lane], g_dig[1][2][lane], g_dig[1][4][lane], 0u);
  const uint32_t sdig = (uint32_t)__cvta_generic_to_shared(sDig);
  const uint32_t szero = (uint32_t)__cvta_generic_to_shared(sZero) + 16u * (uint32_t)(lane & 7);
  const int t0 = 2 * wp;                      // the thread's first plane
  const int pbase = 2 * q + 8 * g + 64 * t0;  // its point pair there (+64 on the second plane)
  double pw = 0.0;
  constexpr float scD = (float)kDScale * 0x1p-20f;  // weight of level 0

  for (int64_t ei = blockIdx.x; ei < E; ei += gridDim.x) {
    const int64_t e = elist ? (int64_t)elist[ei] : ei;  // the element (E: the list's length with a list)
    // ---------------------------------------------------------------- P0: gather, scale, digits of x
    if (tid == 0) prefetch_l2(Gdf + e * 6 * N3, 48u * N3);
    int2 gi[2] = {make_int2(0, 0), make_int2(0, 0)};
    double uv[2][2];  // the thread's inputs, kept for the Helmholtz term and p.w
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (ASSEMBLED) gi[h] = *reinterpret_cast<const int2 *>(l2gm + e * N3 + pbase + 64 * h);
#pragma unroll
    for (int h = 0; h < 2; ++h) load_u<ASSEMBLED>(u, gi[h], e * N3 + pbase + 64 * h, uv[h]);
    int em = max(max(df::exp_field(uv[0][0]), df::exp_field(uv[0][1])),
                 max(df::exp_field(uv[1][0]), df::exp_field(uv[1][1])));
    em = __reduce_max_sync(0xffffffffu, em);
    if (lane == 0) s_red[wp] = em;
    __syncthreads();
    const int su = max(max(s_red[0], s_red[1]), max(s_red[2], s_red[3])) - 1022;  // |u| 2^-su < 1
    float2 xh[2], xl[2];  // x = u 2^-su in double-float
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float2 x0 = df::from_f64_scaled(uv[h][0], su), x1 = df::from_f64_scaled(uv[h][1], su);
      xh[h] = make_float2(x0.x, x1.x);
      xl[h] = make_float2(x0.y, x1.y);
      uint32_t d[NSL];
      digits5(xh[h], xl[h], 1024.0f, 1048576.0f, d);
#pragma unroll
      for (int j = 0; j < NSL; ++j) sDig[dig_word(j, t0 + h, g, q)] = d[j];
    }
    __syncthreads();
    // ---------------------------------------------------------------- P1: ur, us, ut
    contract_pass(sdig, szero, false, FA, FB, scD, wp, lane, sR, sS, sT);
    __syncthreads();
    // ---------------------------------------------------------------- P2: metric
    const float2 *Ge = Gdf + e * 6 * N3;
    int evm = 0;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int p = pbase + 64 * h;
      float2 uh[3], ul[3];
      ld_pair(sR, p, uh[0], ul[0]);
      ld_pair(sS, p, uh[1], ul[1]);
      ld_pair(sT, p, uh[2], ul[2]);
      float2 gh[6], gl[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        const float4 G4 = *reinterpret_cast<const float4 *>(Ge + f * N3 + p);
        gh[f] = make_float2(G4.x, G4.z);
        gl[f] = make_float2(G4.y, G4.w);
      }
      float2 oh, ol;
      metric_row2(gh, gl, 0, 1, 2, uh, ul, oh, ol);
      evm = max(evm, fexp2(oh));
      st_pair(sR, p, oh, ol);
      metric_row2(gh, gl, 1, 3, 4, uh, ul, oh, ol);
      evm = max(evm, fexp2(oh));
      st_pair(sS, p, oh, ol);
      metric_row2(gh, gl, 2, 4, 5, uh, ul, oh, ol);
      evm = max(evm, fexp2(oh));
      st_pair(sT, p, oh, ol);
    }
    evm = __reduce_max_sync(0xffffffffu, evm);
    if (lane == 0) s_red[4 + wp] = evm;
    __syncthreads();
    // digits of v 2^-sv, |v 2^-sv| <= 1: sv = (largest biased exponent) - 126,
    // at least -100 so that the digit scales stay normal binary32 numbers
    // (an element whose v is all zero, or below 2^-100, gives digits of 0)
    const int ev = max(max(s_red[4], s_red[5]), max(s_red[6], s_red[7]));
    const int sv = max(ev - 126, -100);
    const float s1 = pow2f(10 - sv), c2 = pow2f(20 - sv);
    const float scV = pow2f(sv - 15);  // scD 2^sv
    // ---------------------------------------------------------------- P3: transposed contractions
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int t = t0 + h, p = pbase + 64 * h;
      float2 vh, vl;
      uint32_t d[NSL];
      ld_pair(sR, p, vh, vl);
      digits5(vh, vl, s1, c2, d);
#pragma unroll
      for (int j = 0; j < NSL; ++j) sDig[dig_word(j, t, g, q)] = d[j];
      ld_pair(sS, p, vh, vl);
      digits5(vh, vl, s1, c2, d);
#pragma unroll
      for (int j = 0; j < NSL; ++j) sDig[kDigWords + dig_word(j, t, g, q)] = d[j];
      ld_pair(sT, p, vh, vl);
      digits5(vh, vl, s1, c2, d);
#pragma unroll
      for (int j = 0; j < NSL; ++j) sDig[2 * kDigWords + dig_word(j, t, g, q)] = d[j];
    }
    __syncthreads();
    contract_pass(sdig, szero, true, TA, TB, scV, wp, lane, sR, sS, sT);
    __syncthreads();
    // ---------------------------------------------------------------- P4: sum, Helmholtz term, scatter
    dfx::Acc pwe = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int p = pbase + 64 * h;
      float2 ah, al, bh, bl, ch, cl;
      ld_pair(sR, p, ah, al);
      ld_pair(sS, p, bh, bl);
      ld_pair(sT, p, ch, cl);
      // three double-floats summed: TwoSums of the highs, lows added, normalised
      float2 s_, e1, s2, e2, vh, vl;
      dfx::two_sum(ah, bh, s_, e1);
      dfx::two_sum(s_, ch, s2, e2);
      dfx::two_sum(s2, add2(add2(add2(al, bl), cl), add2(e1, e2)), vh, vl);
      if (HELM) {
        const float4 B4 = *reinterpret_cast<const float4 *>(Bdf + e * N3 + p);
        const float2 Bh = make_float2(B4.x, B4.z), Bl = make_float2(B4.y, B4.w);
        dfx::Acc bu = dfx::mul_first(Bh, Bl, xh[h], xl[h]);
        float2 buh, bul;
        dfx::two_sum(bu.s, bu.c, buh, bul);
        dfx::Acc o = dfx::mul_first(dup(h1.x), dup(h1.y), vh, vl);
        dfx::mac(o, dup(h2.x), dup(h2.y), buh, bul);
        dfx::two_sum(o.s, o.c, vh, vl);
      }
      const double v0 = df::to_f64_scaled(vh.x, vl.x, su), v1 = df::to_f64_scaled(vh.y, vl.y, su);
      if (ASSEMBLED) {
        if (wloc) {
          wloc[e * N3 + p] = (gi[h].x >= 0) ? v0 : 0.0;
          wloc[e * N3 + p + 1] = (gi[h].y >= 0) ? v1 : 0.0;
        } else {
          if (gi[h].x >= 0) atomicAdd(&w[gi[h].x], v0);
          if (gi[h].y >= 0) atomicAdd(&w[gi[h].y], v1);
        }
        if (pw_partial != nullptr) dfx::mac(pwe, xh[h], xl[h], vh, vl);
      } else {
        w[e * N3 + p] = v0;
        w[e * N3 + p + 1] = v1;
      }
    }
    if (ASSEMBLED && pw_partial != nullptr) {
      const float2 p0 = df::norm(df::Acc{pwe.s.x, pwe.c.x}), p1 = df::norm(df::Acc{pwe.s.y, pwe.c.y});
      pw += df::to_f64_scaled(p0.x, p0.y, 2 * su) + df::to_f64_scaled(p1.x, p1.y, 2 * su);
    }
    __syncthreads();  // shared tiles and digit planes are reused by the next element
  }
  if (ASSEMBLED && pw_partial != nullptr) {
    double v = pw;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) s_pw[wp] = v;
    __syncthreads();
    // the sum-factorised kernel's count of partials: two per element (one
    // per warp of its 64-thread CTAs); the second slot holds 0
    if (tid == 0) {
      pw_partial[2 * (int64_t)blockIdx.x] = (s_pw[0] + s_pw[1]) + (s_pw[2] + s_pw[3]);
      pw_partial[2 * (int64_t)blockIdx.x + 1] = 0.0;
    }
  }
}

// ---------------------------------------------------------------- register-resident form
// One warp per element, no tiles shared between threads and no barriers.
// Each lane stages only its own words in shared memory (x, then the
// transposed r + s results, and the even-odd forms of wt, per plane pair)
// so that the plane-pair loops can stay rolled: fully unrolled, the code
// outgrew the instruction cache. Lane (g, q) owns the 16 points (i, j, k) =
// (g, 2q + jj, k), jj = 0, 1, k = 0..7: in every k-plane the pair
// (j = 2q, 2q + 1) at row i = g, which is the A-fragment and the
// accumulator layout of the mma, and the whole k-line of both its (i, j)
// columns. Two k-planes k1, k2 = (a, 7 - a) share one mma against a
// block-diagonal operand, so each digit product of a plane pair is one mma
// (and the pair is also the t-line's even-odd output pair):
//   r: A = diag(D_a, D_a), B = the digit planes of x transposed (movmatrix);
//   s: A = diag(X_b(k1), X_b(k2)), B = [D_a^T; D_a^T];
// and the accumulator lands on the lane's own points (rows 0-7 plane k1,
// rows 8-15 plane k2). The t-lines are thread-local: double-float on the
// binary32 pipe, the two columns as the lanes of packed instructions, with
// the even-odd split of D. The transposed r and s contractions of a plane
// pair use one digit scale for wr and ws (their own maximum) and sum into
// one level set; the transposed t-line is added in double-float.
__device__ __forceinline__ int rr_point(int lane, int k, int jj) {
  return (lane >> 2) + 8 * (2 * (lane & 3) + jj) + 64 * k;
}

// Lane-major geometry: per element, plane pair a = (a, 7 - a), c = 2 f + kl
// and lane, one uint4 (hi(jj 0), hi(jj 1), lo(jj 0), lo(jj 1)) of factor f
// at the lane's points of plane a (kl 0) or 7 - a (kl 1); the map as int4 c = (P(2c, 0), P(2c, 1),
// P(2c + 1, 0), P(2c + 1, 1)). Each uint4 load of a warp reads 512
// contiguous bytes.
__global__ void k_tcr_pack(int64_t E, const float2 *__restrict__ Gdf, const int32_t *__restrict__ map,
                           uint4 *__restrict__ Gt, int4 *__restrict__ Mt) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < E * 32; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t >> 5;
    const int lane = (int)(t & 31);
    for (int a = 0; a < 4; ++a)
      for (int f = 0; f < 6; ++f)
        for (int kl = 0; kl < 2; ++kl) {
          const int k = kl ? NP - 1 - a : a;  // the plane pairs are (a, 7 - a)
          const float2 g0 = Gdf[(e * 6 + f) * N3 + rr_point(lane, k, 0)];
          const float2 g1 = Gdf[(e * 6 + f) * N3 + rr_point(lane, k, 1)];
          Gt[((e * 4 + a) * 12 + 2 * f + kl) * 32 + lane] =
              make_uint4(__float_as_uint(g0.x), __float_as_uint(g1.x), __float_as_uint(g0.y), __float_as_uint(g1.y));
        }
    if (map)
      for (int c = 0; c < 4; ++c)
        Mt[(e * 4 + c) * 32 + lane] =
            make_int4(map[e * N3 + rr_point(lane, 2 * c, 0)], map[e * N3 + rr_point(lane, 2 * c, 1)],
                      map[e * N3 + rr_point(lane, 2 * c + 1, 0)], map[e * N3 + rr_point(lane, 2 * c + 1, 1)]);
  }
}

// The t-lines of the lane's two columns (the lanes of packed pairs) with the
// even-odd split of the double-float kernel's line_apply, each lane doing
// its scalar operation sequence: the even and odd forms of a line,
// e_m = x_m + x_{7-m}, o_m = x_m - x_{7-m} (m < 4), then outputs i and
// 7 - i from the 4-term dot products P = A(i, .) e, Q = Bq(i, .) o:
// y_i = P + Q, y_{7-i} = Q - P. The coefficients (hi, hi, lo, lo) come from
// the shared table tq.
__device__ __forceinline__ void eo_form(float2 xmh, float2 xml, float2 xnh, float2 xnl, float2 &eh, float2 &el,
                                        float2 &oh, float2 &ol) {
  float2 s, e;
  dfx::two_sum(xmh, xnh, s, e);
  eh = s;
  el = add2(e, add2(xml, xnl));
  dfx::two_sum(xmh, neg2(xnh), s, e);
  oh = s;
  ol = add2(e, sub2(xml, xnl));
}

template <bool TR>
__device__ __forceinline__ void t_outputs(int i, const float2 (&eh)[4], const float2 (&el)[4], const float2 (&oh)[4],
                                          const float2 (&ol)[4], const float4 (&tq)[2][2][16], float2 &yih,
                                          float2 &yil, float2 &ymh, float2 &yml) {
  const float4 *A = tq[TR ? 1 : 0][0], *Bq = tq[TR ? 1 : 0][1];
  float4 c = A[i * 4];
  dfx::Acc P = dfx::mul_first(make_float2(c.x, c.y), make_float2(c.z, c.w), eh[0], el[0]);
  c = Bq[i * 4];
  dfx::Acc Q = dfx::mul_first(make_float2(c.x, c.y), make_float2(c.z, c.w), oh[0], ol[0]);
#pragma unroll
  for (int m = 1; m < 4; ++m) {
    c = A[i * 4 + m];
    dfx::mac(P, make_float2(c.x, c.y), make_float2(c.z, c.w), eh[m], el[m]);
    c = Bq[i * 4 + m];
    dfx::mac(Q, make_float2(c.x, c.y), make_float2(c.z, c.w), oh[m], ol[m]);
  }
  float2 s, e;
  dfx::two_sum(P.s, Q.s, s, e);
  const float2 t1 = add2(add2(P.c, Q.c), e);
  yih = add2(s, t1);  // Fast2Sum
  yil = sub2(t1, sub2(yih, s));
  dfx::two_sum(Q.s, neg2(P.s), s, e);
  const float2 t2 = add2(sub2(Q.c, P.c), e);
  ymh = add2(s, t2);
  yml = sub2(t2, sub2(ymh, s));
}

// L += A B (m16n8k16, fp16 digits, exact binary32 level sums)
__device__ __forceinline__ void mma_acc(float4 &L, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                        uint32_t b1) {
  mma16(L.x, L.y, L.z, L.w, a0, a1, a2, a3, b0, b1, L.x, L.y, L.z, L.w);
}

// transpose of the 8x8 fp16 matrix whose row g, cols 2q, 2q+1 this lane holds
__device__ __forceinline__ uint32_t trans8(uint32_t a) {
  uint32_t d;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(d) : "r"(a));
  return d;
}

// The Poisson operator (h1 = 1, h2 = 0) in the register-resident form,
// local (E-vectors) or assembled (map through the lane-major copy Mt), with
// the p.w partial of each element from the energy form u^T A_e u =
// sum (ur wr + us ws + ut wt) over the element's points. One warp per
// element (grid = E / 4 CTAs): the partials are [2e] = the element's, [2e + 1] = 0.
constexpr int kTcrWarpF4 = 2 * 4 * 32 * 2;           // float4 of staging per warp (8 KB: x then r + s, wt)
constexpr int kTcrSmem = 4 * kTcrWarpF4 * 16;          // bytes per CTA (4 warps)

template <bool ASSEMBLED>
__global__ void __launch_bounds__(128, 4)
    k_ax_tcr(int64_t E, const uint4 *__restrict__ Gt, const int4 *__restrict__ Mt, const double *__restrict__ u,
             double *__restrict__ w, double *__restrict__ pw_partial, double *__restrict__ wloc,
             const int *__restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  __shared__ float4 s_tq[2][2][16];
  for (int t = threadIdx.x; t < 64; t += blockDim.x) (&s_tq[0][0][0])[t] = (&c_tq[0][0][0])[t];
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  // per-warp staging, each lane only its own words: x at the plane pairs
  // (then, in the same slot, the transposed r + s results) and the even-odd
  // forms of wt, [pair][lane][2] float4 (hi pair, lo pair)
  extern __shared__ __align__(16) float4 s_stage[];
  float4 *sx = s_stage + wp * kTcrWarpF4, *so = sx, *sw = sx + 4 * 32 * 2;
  uint32_t Fd[NSL], Td[NSL];  // D's digits: (D_j[g][2q], D_j[g][2q+1]) and (D_j[2q][g], D_j[2q+1][g])
#pragma unroll
  for (int j = 0; j < NSL; ++j) {
    Fd[j] = g_dig[0][j][lane];
    Td[j] = g_dig[1][j][lane];
  }
  constexpr float scD = (float)kDScale * 0x1p-20f;  // weight of level 0
  const int64_t e = (int64_t)blockIdx.x * 4 + wp;  // one element per warp
  if (e >= E) return;                              // no barrier follows
  if (lane == 0) prefetch_l2(Gt + e * 4 * 12 * 32, 4 * 12 * 32 * 16);  // the element's 24 KB of geometry
  // P0: gather; the element's scale su (|u| 2^-su < 1)
  double uv[NP][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (ASSEMBLED) {
      const int4 mc = Mt[(e * 4 + c) * 32 + lane];
      uv[2 * c][0] = mc.x >= 0 ? u[mc.x] : 0.0;
      uv[2 * c][1] = mc.y >= 0 ? u[mc.y] : 0.0;
      uv[2 * c + 1][0] = mc.z >= 0 ? u[mc.z] : 0.0;
      uv[2 * c + 1][1] = mc.w >= 0 ? u[mc.w] : 0.0;
    } else {
#pragma unroll
      for (int kl = 0; kl < 2; ++kl)
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) uv[2 * c + kl][jj] = u[e * N3 + rr_point(lane, 2 * c + kl, jj)];
    }
  }
  int em = 0;
#pragma unroll
  for (int k = 0; k < NP; ++k) em = max(em, max(df::exp_field(uv[k][0]), df::exp_field(uv[k][1])));
  const int su = __reduce_max_sync(0xffffffffu, em) - 1022;
  float2 xh[NP], xl[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const float2 x0 = df::from_f64_scaled(uv[k][0], su), x1 = df::from_f64_scaled(uv[k][1], su);
    xh[k] = make_float2(x0.x, x1.x);
    xl[k] = make_float2(x0.y, x1.y);
  }
  float2 xeh[4], xel[4], xoh[4], xol[4];  // even and odd forms of the x k-lines
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    eo_form(xh[m], xl[m], xh[NP - 1 - m], xl[NP - 1 - m], xeh[m], xel[m], xoh[m], xol[m]);
    sx[(m * 32 + lane) * 2] = make_float4(xh[m].x, xh[m].y, xl[m].x, xl[m].y);
    sx[(m * 32 + lane) * 2 + 1] = make_float4(xh[NP - 1 - m].x, xh[NP - 1 - m].y, xl[NP - 1 - m].x, xl[NP - 1 - m].y);
  }
  dfx::Acc pwe = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
  // plane pairs (a, 7 - a): stacked in the mma, and the even-odd output pair of the t-lines
#pragma unroll 1
  for (int a = 0; a < NP / 2; ++a) {
    // forward t at the two planes
    float2 th[2], tl[2];
    t_outputs<false>(a, xeh, xel, xoh, xol, s_tq, th[0], tl[0], th[1], tl[1]);
    // digit planes of x at the two planes: (digit at (g, 2q, k), digit at (g, 2q+1, k))
    uint32_t dx1[NSL], dx2[NSL];
    {
      const float4 p1 = sx[(a * 32 + lane) * 2], p2 = sx[(a * 32 + lane) * 2 + 1];
      digits5(make_float2(p1.x, p1.y), make_float2(p1.z, p1.w), 1024.0f, 1048576.0f, dx1);
      digits5(make_float2(p2.x, p2.y), make_float2(p2.z, p2.w), 1024.0f, 1048576.0f, dx2);
    }
    // forward r: level i + j from D's digit i and x's digit j
    float2 urh[2], url[2], ush[2], usl[2];
    {
      uint32_t b1[NSL], b2[NSL];
#pragma unroll
      for (int j = 0; j < NSL; ++j) {
        b1[j] = trans8(dx1[j]);
        b2[j] = trans8(dx2[j]);
      }
      float4 L[NSL];
#pragma unroll
      for (int l = 0; l < NSL; ++l) L[l] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
      for (int i = 0; i < NSL; ++i)
#pragma unroll
        for (int j = 0; i + j < NSL; ++j) mma_acc(L[i + j], Fd[i], 0u, 0u, Fd[i], b1[j], b2[j]);
      recombine(make_float2(L[0].x, L[0].y), make_float2(L[1].x, L[1].y), make_float2(L[2].x, L[2].y),
                make_float2(L[3].x, L[3].y), make_float2(L[4].x, L[4].y), scD, urh[0], url[0]);
      recombine(make_float2(L[0].z, L[0].w), make_float2(L[1].z, L[1].w), make_float2(L[2].z, L[2].w),
                make_float2(L[3].z, L[3].w), make_float2(L[4].z, L[4].w), scD, urh[1], url[1]);
    }
    // forward s
    {
      float4 L[NSL];
#pragma unroll
      for (int l = 0; l < NSL; ++l) L[l] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
      for (int i = 0; i < NSL; ++i)
#pragma unroll
        for (int j = 0; i + j < NSL; ++j) mma_acc(L[i + j], dx1[j], 0u, 0u, dx2[j], Fd[i], Fd[i]);
      recombine(make_float2(L[0].x, L[0].y), make_float2(L[1].x, L[1].y), make_float2(L[2].x, L[2].y),
                make_float2(L[3].x, L[3].y), make_float2(L[4].x, L[4].y), scD, ush[0], usl[0]);
      recombine(make_float2(L[0].z, L[0].w), make_float2(L[1].z, L[1].w), make_float2(L[2].z, L[2].w),
                make_float2(L[3].z, L[3].w), make_float2(L[4].z, L[4].w), scD, ush[1], usl[1]);
    }
    // metric at the pair's four points; kl 0 is plane a, kl 1 plane 7 - a
    float2 wrh[2], wrl[2], wsh[2], wsl[2], wth[2], wtl[2];
    int ev = 0;
#pragma unroll
    for (int kl = 0; kl < 2; ++kl) {
      float2 gh[6], gl[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        const uint4 G4 = Gt[((e * 4 + a) * 12 + 2 * f + kl) * 32 + lane];
        gh[f] = make_float2(__uint_as_float(G4.x), __uint_as_float(G4.y));
        gl[f] = make_float2(__uint_as_float(G4.z), __uint_as_float(G4.w));
      }
      const float2 uh[3] = {urh[kl], ush[kl], th[kl]}, ul[3] = {url[kl], usl[kl], tl[kl]};
      metric_row2(gh, gl, 0, 1, 2, uh, ul, wrh[kl], wrl[kl]);
      metric_row2(gh, gl, 1, 3, 4, uh, ul, wsh[kl], wsl[kl]);
      metric_row2(gh, gl, 2, 4, 5, uh, ul, wth[kl], wtl[kl]);
      ev = max(ev, max(fexp2(wrh[kl]), fexp2(wsh[kl])));
      if (ASSEMBLED && pw_partial != nullptr) {  // energy form of p.w
        dfx::mac(pwe, uh[0], ul[0], wrh[kl], wrl[kl]);
        dfx::mac(pwe, uh[1], ul[1], wsh[kl], wsl[kl]);
        dfx::mac(pwe, uh[2], ul[2], wth[kl], wtl[kl]);
      }
    }
    {
      float2 eh, el, oh_, ol_;
      eo_form(wth[0], wtl[0], wth[1], wtl[1], eh, el, oh_, ol_);
      sw[(a * 32 + lane) * 2] = make_float4(eh.x, eh.y, el.x, el.y);
      sw[(a * 32 + lane) * 2 + 1] = make_float4(oh_.x, oh_.y, ol_.x, ol_.y);
    }
    // digits of (wr, ws) 2^-sv, |.| <= 1, sv from the plane pair's largest exponent
    const int sv = max(__reduce_max_sync(0xffffffffu, ev) - 126, -100);
    const float s1 = pow2f(10 - sv), c2 = pow2f(20 - sv), scV = pow2f(sv - 15);
    uint32_t dr[2][NSL], ds[2][NSL];
#pragma unroll
    for (int kl = 0; kl < 2; ++kl) {
      digits5(wrh[kl], wrl[kl], s1, c2, dr[kl]);
      digits5(wsh[kl], wsl[kl], s1, c2, ds[kl]);
    }
    // transposed r and s into one level set
    {
      float4 L[NSL];
#pragma unroll
      for (int l = 0; l < NSL; ++l) L[l] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
      for (int j = 0; j < NSL; ++j) {
        const uint32_t t1 = trans8(dr[0][j]), t2 = trans8(dr[1][j]);
#pragma unroll
        for (int i = 0; i + j < NSL; ++i) mma_acc(L[i + j], Td[i], 0u, 0u, Td[i], t1, t2);
      }
#pragma unroll
      for (int i = 0; i < NSL; ++i)
#pragma unroll
        for (int j = 0; i + j < NSL; ++j) mma_acc(L[i + j], ds[0][j], 0u, 0u, ds[1][j], Td[i], Td[i]);
      float2 o1h, o1l, o2h, o2l;
      recombine(make_float2(L[0].x, L[0].y), make_float2(L[1].x, L[1].y), make_float2(L[2].x, L[2].y),
                make_float2(L[3].x, L[3].y), make_float2(L[4].x, L[4].y), scV, o1h, o1l);
      recombine(make_float2(L[0].z, L[0].w), make_float2(L[1].z, L[1].w), make_float2(L[2].z, L[2].w),
                make_float2(L[3].z, L[3].w), make_float2(L[4].z, L[4].w), scV, o2h, o2l);
      so[(a * 32 + lane) * 2] = make_float4(o1h.x, o1h.y, o1l.x, o1l.y);
      so[(a * 32 + lane) * 2 + 1] = make_float4(o2h.x, o2h.y, o2l.x, o2l.y);
    }
  }
  // transposed t-lines pair by pair, the sum, back to binary64, scatter
  float2 weh[4], wel[4], woh[4], wol[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const float4 pe = sw[(m * 32 + lane) * 2], po = sw[(m * 32 + lane) * 2 + 1];
    weh[m] = make_float2(pe.x, pe.y);
    wel[m] = make_float2(pe.z, pe.w);
    woh[m] = make_float2(po.x, po.y);
    wol[m] = make_float2(po.z, po.w);
  }
#pragma unroll 1
  for (int a = 0; a < NP / 2; ++a) {
    float2 yh[2], yl[2];
    t_outputs<true>(a, weh, wel, woh, wol, s_tq, yh[0], yl[0], yh[1], yl[1]);
#pragma unroll
    for (int kl = 0; kl < 2; ++kl) {
      const int k = kl ? NP - 1 - a : a;
      const float4 o4 = so[(a * 32 + lane) * 2 + kl];
      float2 s_, e_, vh, vl;
      dfx::two_sum(make_float2(o4.x, o4.y), yh[kl], s_, e_);
      dfx::two_sum(s_, add2(add2(make_float2(o4.z, o4.w), yl[kl]), e_), vh, vl);
      const double v0 = df::to_f64_scaled(vh.x, vl.x, su), v1 = df::to_f64_scaled(vh.y, vl.y, su);
      const int p0 = rr_point(lane, k, 0), p1 = rr_point(lane, k, 1);
      if (ASSEMBLED) {
        const int4 mc = Mt[(e * 4 + k / 2) * 32 + lane];  // again (cached)
        const int g0 = (k & 1) ? mc.z : mc.x, g1 = (k & 1) ? mc.w : mc.y;
        if (wloc) {
          wloc[e * N3 + p0] = g0 >= 0 ? v0 : 0.0;
          wloc[e * N3 + p1] = g1 >= 0 ? v1 : 0.0;
        } else {
          if (g0 >= 0) atomicAdd(&w[g0], v0);
          if (g1 >= 0) atomicAdd(&w[g1], v1);
        }
      } else {
        w[e * N3 + p0] = v0;
        w[e * N3 + p1] = v1;
      }
    }
  }
  if (ASSEMBLED && pw_partial != nullptr) {
    const float2 pa = df::norm(df::Acc{pwe.s.x, pwe.c.x}), pb = df::norm(df::Acc{pwe.s.y, pwe.c.y});
    double v = df::to_f64_scaled(pa.x, pa.y, 2 * su) + df::to_f64_scaled(pb.x, pb.y, 2 * su);
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) {
      pw_partial[2 * e] = v;
      pw_partial[2 * e + 1] = 0.0;
    }
  }
}

}  // namespace

// Launch the tensor-core operator (N = 7 only): same arguments and results as
// sem_launch_ax_df64 with NP = 8; one CTA per element.
int sem_launch_ax_tc(const sem_mesh *m, double h1, double h2, const double *u, double *w, double *pw_partial,
                     bool assembled, cudaStream_t st, const int32_t *map, const int *skip, const int32_t *elist,
                     int64_t nlist) {
  if (m->n != NP) return sem_fail(SEM_ERR_INVALID_ARG, "tensor-core operator: N = 7 only");
  if (int rc = ensure_digits(m->device)) return rc;
  const int64_t nE = elist ? nlist : m->E;
  const unsigned grid = (unsigned)std::max<int64_t>(nE, 1);
  auto split = [](double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
  };
  const float2 h1d = split(h1), h2d = split(h2);
  const bool helm = !(h1 == 1.0 && h2 == 0.0);
  double *wloc = (assembled && !elist) ? (double *)m->det_w : nullptr;
#define LAUNCH(ASM, HLM) \
  k_ax_tc<ASM, HLM><<<grid, kThreads, 0, st>>>(nE, m->Gdf, m->Bdf, h1d, h2d, u, w, map, pw_partial, wloc, skip, elist)
  if (assembled) {
    if (helm) LAUNCH(true, true);
    else LAUNCH(true, false);
  } else {
    if (helm) LAUNCH(false, true);
    else LAUNCH(false, false);
  }
#undef LAUNCH
  SEM_LAUNCH_CHECK("k_ax_tc");
  if (wloc) return sem_launch_gather_add(m, wloc, w, st);
  return SEM_OK;
}

// Lane-major copies of the register-resident route (made once per mesh).
int sem_tcr_prepare(sem_mesh *m, cudaStream_t st) {
  if (m->n != NP) return sem_fail(SEM_ERR_INVALID_ARG, "tensor-core operator: N = 7 only");
  if (int rc = ensure_digits(m->device)) return rc;
  const size_t gbytes = (size_t)m->E * 4 * 12 * 32 * sizeof(uint4), mbytes = (size_t)m->E * 4 * 32 * sizeof(int4);
  void *Gt = nullptr, *Mt = nullptr;
  cudaError_t e = cudaMalloc(&Gt, std::max<size_t>(gbytes, 16));
  if (e == cudaSuccess) e = cudaMalloc(&Mt, std::max<size_t>(mbytes, 16));
  if (e != cudaSuccess) {
    if (Gt) cudaFree(Gt);
    return sem_cuda_fail(e, "sem_mesh_set_tensor_cores: cudaMalloc (lane-major copies)");
  }
  k_tcr_pack<<<grid_for(m->E * 32, 256), 256, 0, st>>>(m->E, m->Gdf, m->l2gm, (uint4 *)Gt, (int4 *)Mt);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(Gt);
    cudaFree(Mt);
    return sem_cuda_fail(e, "sem_mesh_set_tensor_cores: k_tcr_pack");
  }
  m->Gt = Gt;
  m->Mt = Mt;
  return SEM_OK;
}

int sem_launch_ax_tcr(const sem_mesh *m, const double *u, double *w, double *pw_partial, bool assembled,
                      cudaStream_t st, const int *skip) {
  if (m->n != NP || !m->Gt) return sem_fail(SEM_ERR_INVALID_ARG, "tensor-core operator: no lane-major copies");
  if (int rc = ensure_digits(m->device)) return rc;
  double *wloc = assembled ? (double *)m->det_w : nullptr;
  auto kern = assembled ? k_ax_tcr<true> : k_ax_tcr<false>;
  SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcrSmem));
  // one warp per element (a persistent grid with the next element's u
  // prefetched by cp.async measured slower: 2.97 vs 2.54 ms on 64^3)
  const unsigned grid = (unsigned)std::max<int64_t>((m->E + 3) / 4, 1);
  kern<<<grid, 128, kTcrSmem, st>>>(m->E, (const uint4 *)m->Gt, assembled ? (const int4 *)m->Mt : nullptr, u, w,
                                    assembled ? pw_partial : nullptr, wloc, skip);
  SEM_LAUNCH_CHECK("k_ax_tcr");
  if (wloc) return sem_launch_gather_add(m, wloc, w, st);
  return SEM_OK;
}
