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
// Threads: one element per 64-thread CTA, two warps; lane = 4g + q. A thread
// owns the 8 points r in {2q, 2q+1}, s = g, t in {4w..4w+3} (w = warp). The
// digits of a point pair (2q, 2q+1) at one (s, t) are one f16x2 register,
// which is exactly an mma fragment register:
//   r-contractions: the digits are the A operand (rows = s of two t-planes,
//     k = r), D's digits the B operand; the accumulator lands on the
//     thread's own points;
//   s-contractions: D's digits are A (rows = s_out, two levels stacked in
//     the 16 rows), the digits transposed by movmatrix are B (k = s, n = r);
//     the accumulator lands on the thread's own points;
//   t-contractions: lines (r, s) cross the two warps, so the digits go
//     through shared memory (ldmatrix.trans gives B with k = t, n = r); the
//     results (t_out = g, r = 2q..) go back through shared memory.
// In the transposed pass the r- and s-contractions accumulate into the same
// level registers (both land on the thread's points at the same scale).
//
// Phases per element:
//   P0 gather u, element scale su, digits of x (registers and shared memory)
//   P1 forward contractions (24 mma per warp-level per direction pair) and
//      recombination to double-float: ur, us in registers, ut via shared
//   P2 metric (wr, ws, wt) = G (ur, us, ut) in double-float, to shared
//      memory; element scale sv of the result
//   P3 transposed contractions: r and s into one level set, t via shared
//   P4 sum, Helmholtz term, scale back to binary64, scatter (atomics or the
//      deterministic E-vector), p.w partial
#include <math.h>

#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "sem_df64.cuh"
#include "sem_internal.h"

namespace {

constexpr int NP = 8, N3 = 512;
constexpr int NSL = 5;             // digit slices per operand
constexpr double kDScale = 32.0;   // D is sliced as D / 32
constexpr int kMinBlocks = 8;      // resident 64-thread CTAs per SM the register budget aims at

// D's digits as mma fragment registers, per lane: [0][j][lane] = (D_j[g][2q],
// D_j[g][2q+1]) (forward: B of the r-contraction, A of s and t),
// [1][j][lane] = (D_j[2q][g], D_j[2q+1][g]) (the transposed contractions)
__device__ uint32_t g_dig[2][NSL][32];

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
  if (device < 32) g_dig_ready |= 1u << device;
  return SEM_OK;
}

// ---------------------------------------------------------------- tensor-core primitives
// d += A B, m16n8k16, fp16 inputs, f32 accumulate
__device__ __forceinline__ void mma16(float &d0, float &d1, float &d2, float &d3, uint32_t a0, uint32_t a1,
                                      uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t movtrans(uint32_t a) {
  uint32_t d;
  asm("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(d) : "r"(a));
  return d;
}

// four 8x8 b16 matrices, transposed; row addresses from lanes 8i..8i+7
__device__ __forceinline__ void ldsm4t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr)
               : "memory");
}

__device__ __forceinline__ void ldsm1t(uint32_t addr, uint32_t &r0) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x1.trans.shared.b16 {%0}, [%1];" : "=r"(r0) : "r"(addr) : "memory");
}

__device__ __forceinline__ uint32_t pack_f16(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// Digits of y = (h + l) s1 2^-10 (|y| < 1): s1 = 2^10 2^-scale, c2 = s1 2^10.
// Round to nearest integer by the 1.5 2^23 shift. The low word enters at
// the third digit through an exact Fast2Sum (|r| >= |l c2| unless r = 0: r
// is a multiple of ulp(h) there, and |l| < ulp(h)).
__device__ __forceinline__ void digits5(float h, float l, float s1, float c2, float (&d)[NSL]) {
  const float M = 12582912.0f;
  float t = __fmaf_rn(h, s1, M);
  d[0] = __fsub_rn(t, M);
  float r = __fmaf_rn(h, s1, -d[0]);
  t = __fmaf_rn(r, 1024.0f, M);
  d[1] = __fsub_rn(t, M);
  r = __fmaf_rn(r, 1024.0f, -d[1]);
  const float sm = __fmaf_rn(l, c2, r);
  const float z = __fsub_rn(sm, r);
  const float eps = __fmaf_rn(l, c2, -z);
  t = __fmaf_rn(sm, 1024.0f, M);
  d[2] = __fsub_rn(t, M);
  r = __fmaf_rn(sm, 1024.0f, -d[2]);
  r = __fmaf_rn(eps, 1024.0f, r);
  t = __fmaf_rn(r, 1024.0f, M);
  d[3] = __fsub_rn(t, M);
  r = __fmaf_rn(r, 1024.0f, -d[3]);
  d[4] = __fmul_rn(r, 1024.0f);  // rounded to 11 bits by the fp16 conversion
}

// The five level sums L_0..L_4 (exact integers) of one output, weight
// 2^-10(L+2) times sc, to a normalised double-float (16 binary32 operations).
__device__ __forceinline__ float2 recombine(float L0, float L1, float L2, float L3, float L4, float sc) {
  const float M = 12582912.0f;
  const float v1 = __fmul_rn(L1, 0x1p-10f);
  const float hi1 = __fsub_rn(__fadd_rn(v1, M), M);  // integer part of level 1 (|v1| < 2^22)
  const float fr1 = __fsub_rn(v1, hi1);              // its fraction, exact
  const float A = __fadd_rn(L0, hi1);                // integer below 2^24: exact
  const float B = __fmaf_rn(L2, 0x1p-20f, fr1);      // on the 2^-20 grid, below 2^3: exact
  const float C = __fmaf_rn(L4, 0x1p-10f, L3);       // levels 3, 4 in level-3 units (error < 2^-32)
  const float h = __fadd_rn(A, B);                   // Fast2Sum: exact when |A| >= 8, else A + B is exact
  const float e = __fsub_rn(B, __fsub_rn(h, A));
  const float l = __fmaf_rn(C, 0x1p-30f, e);
  const float H = __fadd_rn(h, l);
  const float Lo = __fsub_rn(l, __fsub_rn(H, h));
  return make_float2(__fmul_rn(H, sc), __fmul_rn(Lo, sc));
}

// 15 digit products of D-as-A contractions: A rows 0..7 and 8..15 are two
// levels, B = (digits j of k 0..7 | digits j' of k 8..15); acc[L][0..1] are
// the two outputs of level L held by this thread.
__device__ __forceinline__ void contract_da(const uint32_t (&Dg)[NSL], const uint32_t (&b)[NSL], float (&acc)[NSL][2]) {
  const uint32_t Z = 0u;
  // L1 | L3
  mma16(acc[1][0], acc[1][1], acc[3][0], acc[3][1], Dg[0], Dg[2], Dg[1], Dg[3], b[1], b[0]);
  // L2 | L4
  mma16(acc[2][0], acc[2][1], acc[4][0], acc[4][1], Dg[0], Dg[2], Dg[1], Dg[3], b[2], b[1]);
  // L3: D0 u3 + D1 u2 | L4: D1 u3
  mma16(acc[3][0], acc[3][1], acc[4][0], acc[4][1], Dg[0], Dg[1], Dg[1], Z, b[3], b[2]);
  // L4: D0 u4 + D4 u0 | L2: D2 u0
  mma16(acc[4][0], acc[4][1], acc[2][0], acc[2][1], Dg[0], Z, Dg[4], Dg[2], b[4], b[0]);
  // L0: D0 u0 | (zero rows)
  mma16(acc[0][0], acc[0][1], acc[1][0], acc[1][1], Dg[0], Z, Z, Z, b[0], b[0]);
}

// 15 digit products of U-as-A contractions: A = digits of two t-planes
// (rows 0..7: plane a, rows 8..15: plane b; a[j] = plane a, c[j] = plane b),
// B = D digits; acc[L][0..1] plane a, acc[L][2..3] plane b.
__device__ __forceinline__ void contract_ua(const uint32_t (&a)[NSL], const uint32_t (&c)[NSL],
                                            const uint32_t (&Dg)[NSL], float (&acc)[NSL][4]) {
  const uint32_t Z = 0u;
#define MMA_UA(L, j, jp, i, ip) \
  mma16(acc[L][0], acc[L][1], acc[L][2], acc[L][3], a[j], c[j], (jp) < 0 ? Z : a[(jp) < 0 ? 0 : (jp)], \
        (jp) < 0 ? Z : c[(jp) < 0 ? 0 : (jp)], Dg[i], (ip) < 0 ? Z : Dg[(ip) < 0 ? 0 : (ip)])
  MMA_UA(0, 0, -1, 0, -1);  // D0 u0
  MMA_UA(1, 1, 0, 0, 1);    // D0 u1 + D1 u0
  MMA_UA(2, 2, 1, 0, 1);    // D0 u2 + D1 u1
  MMA_UA(2, 0, -1, 2, -1);  // D2 u0
  MMA_UA(3, 3, 2, 0, 1);    // D0 u3 + D1 u2
  MMA_UA(3, 1, 0, 2, 3);    // D2 u1 + D3 u0
  MMA_UA(4, 4, 3, 0, 1);    // D0 u4 + D1 u3
  MMA_UA(4, 2, 1, 2, 3);    // D2 u2 + D3 u1
  MMA_UA(4, 0, -1, 4, -1);  // D4 u0
#undef MMA_UA
}

// shared-memory digit planes: slice j, plane t, row s holds the 8 r-values
// (16 bytes) at chunk (j 8 + t) 8 + (s ^ t) (the xor spreads the rows of a
// fixed-s matrix over all bank groups)
__device__ __forceinline__ int dig_word(int j, int t, int s, int q) { return (((j * 8 + t) * 8 + (s ^ t)) << 2) + q; }

__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ float2 metric_row(float2 g0, float2 g1, float2 g2, float2 u0, float2 u1, float2 u2) {
  df::Acc a = df::mul_first(g0.x, g0.y, u0.x, u0.y);
  df::mac(a, g1.x, g1.y, u1.x, u1.y);
  df::mac(a, g2.x, g2.y, u2.x, u2.y);
  float h, l;
  df::fast_two_sum(a.s, a.c, h, l);
  return make_float2(h, l);
}

__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((unsigned)(k + 127) << 23); }

// largest biased binary32 exponent of the hi parts (NaN/inf excluded)
__device__ __forceinline__ int fexp(float h) {
  const int e = (int)((__float_as_uint(h) >> 23) & 0xFFu);
  return e == 0xFF ? 0 : e;
}

// the two inputs of a point pair: gathered through the map (assembled), or
// from the caller's E-vector (only 8-byte alignment is promised there)
template <bool ASSEMBLED>
__device__ __forceinline__ void load_u(const double *__restrict__ u, const int32_t (&gi)[2], int64_t l, double (&v)[2]) {
  if (ASSEMBLED) {
    v[0] = gi[0] >= 0 ? u[gi[0]] : 0.0;
    v[1] = gi[1] >= 0 ? u[gi[1]] : 0.0;
  } else {
    v[0] = u[l];
    v[1] = u[l + 1];
  }
}

template <bool ASSEMBLED, bool HELM>
__global__ void __launch_bounds__(64, kMinBlocks)
    k_ax_tc(int64_t E, const float2 *__restrict__ Gdf, const float2 *__restrict__ Bdf, float2 h1, float2 h2,
            const double *__restrict__ u, double *__restrict__ w, const int32_t *__restrict__ l2gm,
            double *__restrict__ pw_partial, double *__restrict__ wloc, const int *__restrict__ skip,
            const int32_t *__restrict__ elist) {
  if (skip != nullptr && *skip != 0) return;
  __shared__ __align__(16) float2 sR[N3];
  __shared__ __align__(16) float2 sS[N3];
  __shared__ __align__(16) float2 sT[N3];
  __shared__ __align__(16) uint32_t sDig[NSL * 256];
  __shared__ int s_red[4];
  __shared__ double s_pw[2];
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31, g = lane >> 2, q = lane & 3;
  uint32_t Fd[NSL], Td[NSL];
#pragma unroll
  for (int j = 0; j < NSL; ++j) {
    Fd[j] = g_dig[0][j][lane];
    Td[j] = g_dig[1][j][lane];
  }
  const uint32_t sdig_base = (uint32_t)__cvta_generic_to_shared(sDig);
  // ldmatrix row addresses: lane L reads row t = L & 7 of matrix L >> 3
  const int lrow = lane & 7, lmat = lane >> 3;
  double pw = 0.0;
  const float scD = (float)kDScale * 0x1p-20f;  // weight of level 0

  for (int64_t ei = blockIdx.x; ei < E; ei += gridDim.x) {
    const int64_t e = elist ? (int64_t)elist[ei] : ei;  // the element (E: the list's length with a list)
    // ---------------------------------------------------------------- P0
    if (tid == 0) prefetch_l2(Gdf + e * 6 * N3, 48u * N3);
    int32_t gi[4][2];
#pragma unroll
    for (int tt = 0; tt < 4; ++tt) {
      const int p = 2 * q + 8 * g + 64 * (4 * wp + tt);
      if (ASSEMBLED) {
        const int2 ii = *reinterpret_cast<const int2 *>(l2gm + e * N3 + p);
        gi[tt][0] = ii.x;
        gi[tt][1] = ii.y;
      }
    }
    double uv0[4][2];  // the thread's inputs (read again from L2 in P4)
#pragma unroll
    for (int tt = 0; tt < 4; ++tt) {
      const int p = 2 * q + 8 * g + 64 * (4 * wp + tt);
      load_u<ASSEMBLED>(u, gi[tt], e * N3 + p, uv0[tt]);
    }
    int em = 0;
#pragma unroll
    for (int tt = 0; tt < 4; ++tt) em = max(em, max(df::exp_field(uv0[tt][0]), df::exp_field(uv0[tt][1])));
    em = __reduce_max_sync(0xffffffffu, em);
    if (lane == 0) s_red[wp] = em;
    __syncthreads();
    const int su = max(s_red[0], s_red[1]) - 1022;  // |u| 2^-su < 1
    // digits of the thread's point pairs, one f16x2 word per (slice, plane),
    // kept in shared memory: the owner reads its own words back per plane
#pragma unroll
    for (int tt = 0; tt < 4; ++tt) {
      float d0[NSL], d1[NSL];
      const float2 x0 = df::from_f64_scaled(uv0[tt][0], su), x1 = df::from_f64_scaled(uv0[tt][1], su);
      digits5(x0.x, x0.y, 1024.0f, 1048576.0f, d0);
      digits5(x1.x, x1.y, 1024.0f, 1048576.0f, d1);
      const int t = 4 * wp + tt;
#pragma unroll
      for (int j = 0; j < NSL; ++j) sDig[dig_word(j, t, g, q)] = pack_f16(d0[j], d1[j]);
    }
    __syncthreads();
    // ---------------------------------------------------------------- P1
    // r: U-as-A over the plane pairs (4w, 4w+1), (4w+2, 4w+3); ur -> sR, us -> sS
    // (own points), ut -> sT (points of other threads)
#pragma unroll 1
    for (int pp = 0; pp < 2; ++pp) {
      float acc[NSL][4];
#pragma unroll
      for (int L = 0; L < NSL; ++L) acc[L][0] = acc[L][1] = acc[L][2] = acc[L][3] = 0.0f;
      uint32_t a[NSL], c[NSL];
      const int ta = 4 * wp + 2 * pp;
#pragma unroll
      for (int j = 0; j < NSL; ++j) {
        a[j] = sDig[dig_word(j, ta, g, q)];
        c[j] = sDig[dig_word(j, ta + 1, g, q)];
      }
      contract_ua(a, c, Fd, acc);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = 2 * q + 8 * g + 64 * (4 * wp + 2 * pp + h);
        const float2 o0 = recombine(acc[0][2 * h], acc[1][2 * h], acc[2][2 * h], acc[3][2 * h], acc[4][2 * h], scD);
        const float2 o1 =
            recombine(acc[0][2 * h + 1], acc[1][2 * h + 1], acc[2][2 * h + 1], acc[3][2 * h + 1], acc[4][2 * h + 1], scD);
        *reinterpret_cast<float4 *>(&sR[p]) = make_float4(o0.x, o0.y, o1.x, o1.y);
      }
    }
    // s: D-as-A per plane, B = the transposed digit matrices
#pragma unroll 1
    for (int tt = 0; tt < 4; ++tt) {
      float acc[NSL][2];
#pragma unroll
      for (int L = 0; L < NSL; ++L) acc[L][0] = acc[L][1] = 0.0f;
      uint32_t b[NSL];
#pragma unroll
      for (int j = 0; j < NSL; ++j) b[j] = movtrans(sDig[dig_word(j, 4 * wp + tt, g, q)]);
      contract_da(Fd, b, acc);
      const int p = 2 * q + 8 * g + 64 * (4 * wp + tt);
      const float2 o0 = recombine(acc[0][0], acc[1][0], acc[2][0], acc[3][0], acc[4][0], scD);
      const float2 o1 = recombine(acc[0][1], acc[1][1], acc[2][1], acc[3][1], acc[4][1], scD);
      *reinterpret_cast<float4 *>(&sS[p]) = make_float4(o0.x, o0.y, o1.x, o1.y);
    }
    // t: D-as-A per s (this warp: s = 4w..4w+3), B from shared memory
#pragma unroll 1
    for (int ss = 0; ss < 4; ++ss) {
      const int s = 4 * wp + ss;
      uint32_t b[NSL];
      ldsm4t(sdig_base + 4u * (uint32_t)dig_word(lmat, lrow, s, 0), b[0], b[1], b[2], b[3]);
      ldsm1t(sdig_base + 4u * (uint32_t)dig_word(4, lrow, s, 0), b[4]);
      float acc[NSL][2];
#pragma unroll
      for (int L = 0; L < NSL; ++L) acc[L][0] = acc[L][1] = 0.0f;
      contract_da(Fd, b, acc);
      // outputs (t_out = g, r = 2q, 2q+1) at this s
      const float2 o0 = recombine(acc[0][0], acc[1][0], acc[2][0], acc[3][0], acc[4][0], scD);
      const float2 o1 = recombine(acc[0][1], acc[1][1], acc[2][1], acc[3][1], acc[4][1], scD);
      *reinterpret_cast<float4 *>(&sT[2 * q + 8 * s + 64 * g]) = make_float4(o0.x, o0.y, o1.x, o1.y);
    }
    __syncthreads();
    // ---------------------------------------------------------------- P2
    const float2 *Ge = Gdf + e * 6 * N3;
    int evm = 0;
#pragma unroll 1
    for (int tt = 0; tt < 4; ++tt) {
      const int p = 2 * q + 8 * g + 64 * (4 * wp + tt);
      const float4 ur4 = *reinterpret_cast<const float4 *>(&sR[p]);
      const float4 us4 = *reinterpret_cast<const float4 *>(&sS[p]);
      const float4 ut4 = *reinterpret_cast<const float4 *>(&sT[p]);
      const float2 ur[2] = {make_float2(ur4.x, ur4.y), make_float2(ur4.z, ur4.w)};
      const float2 us[2] = {make_float2(us4.x, us4.y), make_float2(us4.z, us4.w)};
      const float2 ut[2] = {make_float2(ut4.x, ut4.y), make_float2(ut4.z, ut4.w)};
      float4 G4[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) G4[f] = *reinterpret_cast<const float4 *>(Ge + f * N3 + p);
      float2 vr[2], vs[2], vt[2];
#pragma unroll
      for (int o = 0; o < 2; ++o) {
        float2 gg[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) gg[f] = o == 0 ? make_float2(G4[f].x, G4[f].y) : make_float2(G4[f].z, G4[f].w);
        vr[o] = metric_row(gg[0], gg[1], gg[2], ur[o], us[o], ut[o]);
        vs[o] = metric_row(gg[1], gg[3], gg[4], ur[o], us[o], ut[o]);
        vt[o] = metric_row(gg[2], gg[4], gg[5], ur[o], us[o], ut[o]);
        evm = max(evm, max(fexp(vr[o].x), max(fexp(vs[o].x), fexp(vt[o].x))));
      }
      *reinterpret_cast<float4 *>(&sR[p]) = make_float4(vr[0].x, vr[0].y, vr[1].x, vr[1].y);
      *reinterpret_cast<float4 *>(&sS[p]) = make_float4(vs[0].x, vs[0].y, vs[1].x, vs[1].y);
      *reinterpret_cast<float4 *>(&sT[p]) = make_float4(vt[0].x, vt[0].y, vt[1].x, vt[1].y);
    }
    evm = __reduce_max_sync(0xffffffffu, evm);
    if (lane == 0) s_red[2 + wp] = evm;
    __syncthreads();
    // digits of v 2^-sv, |v 2^-sv| <= 1: sv = (largest biased exponent) - 126,
    // at least -100 so that the digit scales stay normal binary32 numbers
    // (an element whose v is all zero, or below 2^-100, gives digits of 0)
    const int ev = max(s_red[2], s_red[3]);
    const int sv = max(ev - 126, -100);
    const float s1 = pow2f(10 - sv), c2 = pow2f(20 - sv);
    const float scV = pow2f(sv - 15);  // scD 2^sv
    // ---------------------------------------------------------------- P3
    // t first: digits of wt to shared memory (the forward digits are no longer needed)
#pragma unroll
    for (int tt = 0; tt < 4; ++tt) {
      const int t = 4 * wp + tt, p = 2 * q + 8 * g + 64 * t;
      const float4 v4 = *reinterpret_cast<const float4 *>(&sT[p]);
      float d0[NSL], d1[NSL];
      digits5(v4.x, v4.y, s1, c2, d0);
      digits5(v4.z, v4.w, s1, c2, d1);
#pragma unroll
      for (int j = 0; j < NSL; ++j) sDig[dig_word(j, t, g, q)] = pack_f16(d0[j], d1[j]);
    }
    // r and s into one level set, per plane pair
#pragma unroll 1
    for (int pp = 0; pp < 2; ++pp) {
      float acc[NSL][4];
#pragma unroll
      for (int L = 0; L < NSL; ++L) acc[L][0] = acc[L][1] = acc[L][2] = acc[L][3] = 0.0f;
      uint32_t a[NSL], c[NSL];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int t = 4 * wp + 2 * pp + h, p = 2 * q + 8 * g + 64 * t;
        const float4 r4 = *reinterpret_cast<const float4 *>(&sR[p]);
        const float4 s4 = *reinterpret_cast<const float4 *>(&sS[p]);
        float d0[NSL], d1[NSL];
        digits5(r4.x, r4.y, s1, c2, d0);
        digits5(r4.z, r4.w, s1, c2, d1);
#pragma unroll
        for (int j = 0; j < NSL; ++j) (h == 0 ? a[j] : c[j]) = pack_f16(d0[j], d1[j]);
        digits5(s4.x, s4.y, s1, c2, d0);
        digits5(s4.z, s4.w, s1, c2, d1);
        uint32_t b[NSL];
#pragma unroll
        for (int j = 0; j < NSL; ++j) b[j] = movtrans(pack_f16(d0[j], d1[j]));
        // s: D^T as A, the two outputs of plane t land in acc[.][2h], acc[.][2h+1]
        float sacc[NSL][2];
#pragma unroll
        for (int L = 0; L < NSL; ++L) {
          sacc[L][0] = acc[L][2 * h];
          sacc[L][1] = acc[L][2 * h + 1];
        }
        contract_da(Td, b, sacc);
#pragma unroll
        for (int L = 0; L < NSL; ++L) {
          acc[L][2 * h] = sacc[L][0];
          acc[L][2 * h + 1] = sacc[L][1];
        }
      }
      contract_ua(a, c, Td, acc);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int t = 4 * wp + 2 * pp + h, p = 2 * q + 8 * g + 64 * t;
        const float2 o0 = recombine(acc[0][2 * h], acc[1][2 * h], acc[2][2 * h], acc[3][2 * h], acc[4][2 * h], scV);
        const float2 o1 =
            recombine(acc[0][2 * h + 1], acc[1][2 * h + 1], acc[2][2 * h + 1], acc[3][2 * h + 1], acc[4][2 * h + 1], scV);
        *reinterpret_cast<float4 *>(&sR[p]) = make_float4(o0.x, o0.y, o1.x, o1.y);
      }
    }
    __syncthreads();  // the digits of wt are in shared memory; sT is free
#pragma unroll 1
    for (int ss = 0; ss < 4; ++ss) {
      const int s = 4 * wp + ss;
      uint32_t b[NSL];
      ldsm4t(sdig_base + 4u * (uint32_t)dig_word(lmat, lrow, s, 0), b[0], b[1], b[2], b[3]);
      ldsm1t(sdig_base + 4u * (uint32_t)dig_word(4, lrow, s, 0), b[4]);
      float acc[NSL][2];
#pragma unroll
      for (int L = 0; L < NSL; ++L) acc[L][0] = acc[L][1] = 0.0f;
      contract_da(Td, b, acc);
      const float2 o0 = recombine(acc[0][0], acc[1][0], acc[2][0], acc[3][0], acc[4][0], scV);
      const float2 o1 = recombine(acc[0][1], acc[1][1], acc[2][1], acc[3][1], acc[4][1], scV);
      *reinterpret_cast<float4 *>(&sT[2 * q + 8 * s + 64 * g]) = make_float4(o0.x, o0.y, o1.x, o1.y);
    }
    __syncthreads();
    // ---------------------------------------------------------------- P4
    df::Acc pwe = {0.0f, 0.0f};
#pragma unroll 1
    for (int tt = 0; tt < 4; ++tt) {
      const int p = 2 * q + 8 * g + 64 * (4 * wp + tt);
      const float4 a4 = *reinterpret_cast<const float4 *>(&sR[p]);
      const float4 b4 = *reinterpret_cast<const float4 *>(&sT[p]);
      float2 Bv2[2];
      if (HELM) {
        const float4 B4 = *reinterpret_cast<const float4 *>(Bdf + e * N3 + p);
        Bv2[0] = make_float2(B4.x, B4.y);
        Bv2[1] = make_float2(B4.z, B4.w);
      }
      int32_t gp[2] = {0, 0};  // the point pair's gather indices, read again (L1/L2)
      if (ASSEMBLED) {
        const int2 ii = *reinterpret_cast<const int2 *>(l2gm + e * N3 + p);
        gp[0] = ii.x;
        gp[1] = ii.y;
      }
      double uv[2];
      if (HELM || (ASSEMBLED && pw_partial != nullptr)) load_u<ASSEMBLED>(u, gp, e * N3 + p, uv);
#pragma unroll
      for (int o = 0; o < 2; ++o) {
        df::Acc acc = {o == 0 ? a4.x : a4.z, o == 0 ? a4.y : a4.w};
        df::acc_add(acc, o == 0 ? b4.x : b4.z, o == 0 ? b4.y : b4.w);
        float2 v = df::norm(acc);
        float2 xk = make_float2(0.0f, 0.0f);
        if (HELM || (ASSEMBLED && pw_partial != nullptr)) xk = df::from_f64_scaled(uv[o], su);
        if (HELM) {
          const float2 buv = df::norm(df::mul_first(Bv2[o].x, Bv2[o].y, xk.x, xk.y));
          df::Acc oo = df::mul_first(h1.x, h1.y, v.x, v.y);
          df::mac(oo, h2.x, h2.y, buv.x, buv.y);
          v = df::norm(oo);
        }
        const double vd = df::to_f64_scaled(v.x, v.y, su);
        if (ASSEMBLED) {
          const int32_t gg = gp[o];
          if (wloc) wloc[e * N3 + p + o] = (gg >= 0) ? vd : 0.0;
          else if (gg >= 0) atomicAdd(&w[gg], vd);
          if (pw_partial != nullptr) df::mac(pwe, xk.x, xk.y, v.x, v.y);
        } else {
          w[e * N3 + p + o] = vd;
        }
      }
    }
    if (ASSEMBLED && pw_partial != nullptr) {
      const float2 pn = df::norm(pwe);
      pw += df::to_f64_scaled(pn.x, pn.y, 2 * su);
    }
    __syncthreads();  // shared tiles and digit planes are reused by the next element
  }
  if (ASSEMBLED && pw_partial != nullptr) {
    double v = pw;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) s_pw[wp] = v;
    __syncthreads();
    if (tid == 0) pw_partial[blockIdx.x] = s_pw[0] + s_pw[1];
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
  k_ax_tc<ASM, HLM><<<grid, 64, 0, st>>>(nE, m->Gdf, m->Bdf, h1d, h2d, u, w, map, pw_partial, wloc, skip, elist)
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
