// binary64-accurate matrix-free Helmholtz operator in double-float
// arithmetic on the binary32 pipe (same operator as sem_ax.cu, Sec. 2.2).
//
// Why: on GB300 binary64 FMA runs at ~1.2 TFLOP/s against ~74 TFLOP/s for
// binary32, so the native-FP64 operator is bound by the FP64 pipe at about
// ten times the HBM time. Carrying every value as hi + lo binary32 with
// error-free transformations costs ~10 binary32 operations per binary64
// multiply-add and keeps ~2^-46 relative accuracy.
//
// Structure per element (NP = N+1 points per direction, NP^2 threads; one
// element per CTA at N = 7, one CTA per element group in every launch):
//   P0  gather the t-column u(a,b,:) (binary64; all indices, then all
//       values), split to df64 into the shared tile U; thread 0 starts the
//       L2 prefetch of the element's geometric factors
//   P1  each thread contracts three lines with D, one loop body: the r-line
//       u(:,a,b) -> R, the s-line u(a,:,b) -> S, its t-line -> T (T is the
//       U tile, written after a barrier; u stays in the thread's registers)
//   P2  pointwise metric on its t-column: (wr, ws, wt) = G (ur, us, ut), the
//       factors of level k + 1 loaded while level k is computed
//   P3  transposed contractions of the same lines, in place
//   P4  w(a,b,:) = T + R + S, then h1 w + h2 B u, back to binary64, scatter
// The 1-D contractions use the even-odd split of the centro-antisymmetric
// D (D[N-i][N-j] = -D[i][j]), which halves the multiply-adds; for even NP
// the even and the odd dot product of each output pair run as the two lanes
// of packed f32x2 instructions (bit-identical to the scalar sequence).
#include <algorithm>
#include <mutex>
#include <vector>

#include "sem_df64.cuh"
#include "sem_df64x2.cuh"
#include "sem_internal.h"

namespace {

// ---------------------------------------------------------------- tables
// Per NP: even NP -> A, Bq for D and for D^T (4 (NP/2)^2 entries);
// odd NP -> D and D^T in full (2 NP^2 entries). Entries are (hi, lo).
__host__ __device__ constexpr int tab_size(int np) { return (np % 2 == 0) ? np * np : 2 * np * np; }
__host__ __device__ constexpr int tab_off(int np) { return np <= 2 ? 0 : tab_off(np - 1) + tab_size(np - 1); }
constexpr int kTabTotal = tab_off(SEM_MAXNP + 1);

__constant__ float2 c_tab[kTabTotal];

std::mutex g_tab_mu;
unsigned g_tab_ready = 0;  // bit per device

float2 split_host(double v) {
  float hi = (float)v;
  float lo = (float)(v - (double)hi);
  return make_float2(hi, lo);
}

int ensure_tables(int device) {
  std::lock_guard<std::mutex> lk(g_tab_mu);
  if (device < 32 && (g_tab_ready >> device) & 1u) return SEM_OK;
  std::vector<float2> tab(kTabTotal);
  for (int np = 2; np <= SEM_MAXNP; ++np) {
    const int N = np - 1;
    double xi[SEM_MAXNP], rho[SEM_MAXNP], D[SEM_MAXNP * SEM_MAXNP];
    if (int rc = sem_gll_host(N, xi, rho, D)) return rc;
    float2 *t = tab.data() + tab_off(np);
    if (np % 2 == 0) {
      const int h = np / 2;
      for (int tr = 0; tr < 2; ++tr) {  // tr = 1: D^T
        auto M = [&](int i, int j) { return tr ? D[j * np + i] : D[i * np + j]; };
        float2 *A = t + tr * 2 * h * h, *Bq = A + h * h;
        for (int i = 0; i < h; ++i)
          for (int m = 0; m < h; ++m) {
            A[i * h + m] = split_host(0.5 * (M(i, m) + M(i, N - m)));
            Bq[i * h + m] = split_host(0.5 * (M(i, m) - M(i, N - m)));
          }
      }
    } else {
      for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) {
          t[i * np + j] = split_host(D[i * np + j]);
          t[np * np + i * np + j] = split_host(D[j * np + i]);
        }
    }
  }
  SEM_CUDA(cudaMemcpyToSymbol(c_tab, tab.data(), sizeof(float2) * kTabTotal));
  if (device < 32) g_tab_ready |= 1u << device;
  return SEM_OK;
}

// Shared coefficient table of the even-odd split (even NP): entry [i H + m]
// = (A.hi, Bq.hi, A.lo, Bq.lo) for D, then the same for D^T at H^2, so one
// 128-bit load feeds both packed lanes of a multiply-add.
template <int NP>
struct KqSize {
  static constexpr int value = (NP % 2 == 0) ? NP * NP / 2 : 1;
};


template <int NP>
__device__ __forceinline__ void load_kq(float4 *kq) {
  if constexpr (NP % 2 == 0) {
    constexpr int H = NP / 2;
    for (int q = threadIdx.x; q < 2 * H * H; q += blockDim.x) {
      const int tr = q / (H * H), im = q - tr * H * H;
      const float2 *A = c_tab + tab_off(NP) + tr * 2 * H * H;
      const float2 a = A[im], b = A[H * H + im];
      kq[q] = make_float4(a.x, b.x, a.y, b.y);
    }
  }
}

// y = M x along one line (M = D, or D^T when TR), df64 in, normalised df64
// out. Compensated dot products (exact products, TwoSum accumulation).
template <int NP, bool TR>
__device__ __forceinline__ void line_apply(const float2 (&x)[NP], float2 (&y)[NP]) {
  constexpr int N = NP - 1;
  if constexpr (NP % 2 == 0) {
    constexpr int H = NP / 2;
    const float2 *A = c_tab + tab_off(NP) + (TR ? 2 * H * H : 0);
    const float2 *Bq = A + H * H;
    float2 xe[H], xo[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
      float s, e;
      df::two_sum(x[m].x, x[N - m].x, s, e);
      xe[m] = make_float2(s, df::add(e, df::add(x[m].y, x[N - m].y)));
      df::two_sum(x[m].x, -x[N - m].x, s, e);
      xo[m] = make_float2(s, df::add(e, df::sub(x[m].y, x[N - m].y)));
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
      df::Acc P = df::mul_first(A[i * H].x, A[i * H].y, xe[0].x, xe[0].y);
      df::Acc Q = df::mul_first(Bq[i * H].x, Bq[i * H].y, xo[0].x, xo[0].y);
#pragma unroll
      for (int m = 1; m < H; ++m) {
        df::mac(P, A[i * H + m].x, A[i * H + m].y, xe[m].x, xe[m].y);
        df::mac(Q, Bq[i * H + m].x, Bq[i * H + m].y, xo[m].x, xo[m].y);
      }
      float s, e, h, l;
      df::two_sum(P.s, Q.s, s, e);
      df::fast_two_sum(s, df::add(df::add(P.c, Q.c), e), h, l);
      y[i] = make_float2(h, l);
      df::two_sum(Q.s, -P.s, s, e);
      df::fast_two_sum(s, df::add(df::sub(Q.c, P.c), e), h, l);
      y[N - i] = make_float2(h, l);
    }
  } else {
    const float2 *M = c_tab + tab_off(NP) + (TR ? NP * NP : 0);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      df::Acc a = df::mul_first(M[i * NP].x, M[i * NP].y, x[0].x, x[0].y);
#pragma unroll
      for (int m = 1; m < NP; ++m) df::mac(a, M[i * NP + m].x, M[i * NP + m].y, x[m].x, x[m].y);
      float h, l;
      df::fast_two_sum(a.s, a.c, h, l);
      y[i] = make_float2(h, l);
    }
  }
}

// The same contraction for even NP, writing its outputs straight to the
// shared tile O at base + str m. The even and the odd dot product of each
// output pair run as the two lanes of packed f32x2 instructions with
// coefficients (A.hi, Bq.hi, A.lo, Bq.lo) from kq, and so do the folding of
// the inputs (sum and difference of x_m and x_{N-m}) and the final sums of
// each output pair (P + Q and Q - P). Each lane does exactly the operation
// sequence of line_apply, so the results are bit-identical to it. The output
// loop is rolled pairwise to bound the live registers.
template <int NP, bool TR>
__device__ __forceinline__ void line_apply_store(const float2 (&x)[NP], float2 *O, int base, int str,
                                                 const float4 *__restrict__ kq) {
  static_assert(NP % 2 == 0, "even-odd form");
  constexpr int N = NP - 1, H = NP / 2;
  const float4 *K = kq + (TR ? H * H : 0);
  float2 eh[H], el[H];
#pragma unroll
  for (int m = 0; m < H; ++m) {  // lane x: x_m + x_{N-m}, lane y: x_m - x_{N-m}
    const float2 xn = make_float2(x[N - m].x, -x[N - m].x);
    dfx::two_sum(make_float2(x[m].x, x[m].x), xn, eh[m], el[m]);
    el[m] = dfx::add(el[m], dfx::add(make_float2(x[m].y, x[m].y), make_float2(x[N - m].y, -x[N - m].y)));
  }
#pragma unroll 2
  for (int i = 0; i < H; ++i) {
    float4 k = K[i * H];
    dfx::Acc PQ = dfx::mul_first(make_float2(k.x, k.y), make_float2(k.z, k.w), eh[0], el[0]);
#pragma unroll
    for (int m = 1; m < H; ++m) {
      k = K[i * H + m];
      dfx::mac(PQ, make_float2(k.x, k.y), make_float2(k.z, k.w), eh[m], el[m]);
    }
    // lane x: output i = P + Q, lane y: output N - i = Q - P
    float2 s, e;
    dfx::two_sum(PQ.s, make_float2(PQ.s.y, -PQ.s.x), s, e);
    const float2 c = dfx::add(dfx::add(PQ.c, make_float2(PQ.c.y, -PQ.c.x)), e);
    const float2 h = dfx::add(s, c);
    const float2 l = dfx::sub(c, dfx::sub(h, s));  // Fast2Sum
    O[base + str * i] = make_float2(h.x, l.x);
    O[base + str * (N - i)] = make_float2(h.y, l.y);
  }
}

// L2 prefetch of a contiguous block (bytes a multiple of 16, 16-byte aligned)
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// one output of the metric step: g0 u0 + g1 u1 + g2 u2
__device__ __forceinline__ float2 metric_row(float2 g0, float2 g1, float2 g2, float2 u0, float2 u1, float2 u2) {
  df::Acc a = df::mul_first(g0.x, g0.y, u0.x, u0.y);
  df::mac(a, g1.x, g1.y, u1.x, u1.y);
  df::mac(a, g2.x, g2.y, u2.x, u2.y);
  float h, l;
  df::fast_two_sum(a.s, a.c, h, l);
  return make_float2(h, l);
}

template <int NP>
struct DfCfg {
  static constexpr int N2 = NP * NP;
  static constexpr int N3 = NP * NP * NP;
  static constexpr int PJ = NP + 1;        // padded r-line stride (avoids bank conflicts)
  static constexpr int PK = NP * (NP + 1);
  static constexpr int TILE = NP * PK;     // float2 per tile
  // at least 128 threads per CTA, shared tiles within 48 KB
  static constexpr int ELB_T = (N2 >= 128) ? 1 : 128 / N2;
  static constexpr int ELB_S = (48 * 1024) / (4 * NP * NP * (NP + 1) * (int)sizeof(float2));
  // NP = 8: one element (64 threads) per CTA, so barriers wait on two warps only
  static constexpr int ELB = (NP == 8) ? 1 : (ELB_T < ELB_S ? ELB_T : (ELB_S > 0 ? ELB_S : 1));
  static constexpr int THREADS = N2 * ELB;
  // the operator: tiles U, R, S; the t-derivative T replaces U once every
  // thread has read its r/s lines (the Helmholtz term takes u from the
  // thread's own registers). The same for both forms.
  static constexpr int smem_ax(bool) { return 3 * TILE * ELB * (int)sizeof(float2); }
  // NP = 8: twelve 64-thread CTAs per SM (at most 85 registers per thread)
  static constexpr int MINB = (NP == 8) ? 12 : 1;
  // p.w partial sums per CTA: one per warp when the CTA is whole warps (a
  // shuffle tree each, no CTA barrier), else one per CTA
  static constexpr int PW_PARTS = (THREADS % 32 == 0) ? THREADS / 32 : 1;
};

template <int NP, bool ASSEMBLED, bool HELM>
__global__ void __launch_bounds__(DfCfg<NP>::THREADS, DfCfg<NP>::MINB)
    k_ax_df64(int64_t E, const float2 *__restrict__ Gdf, const float2 *__restrict__ Bdf, float2 h1, float2 h2,
              const double *__restrict__ u, double *__restrict__ w, const int32_t *__restrict__ l2gm,
              double *__restrict__ pw_partial, double *__restrict__ wloc, const int *__restrict__ skip,
              const int32_t *__restrict__ elist) {
  using C = DfCfg<NP>;
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ float2 sm2[];
  __shared__ float4 kq[KqSize<NP>::value];  // read after the first barrier of the element loop
  load_kq<NP>(kq);
  const int tid = threadIdx.x;
  const int le = tid / C::N2;
  const int t = tid - le * C::N2;
  const int a = t % NP, b = t / NP;
  constexpr int NT = 3;  // tiles per element
  float2 *U = sm2 + le * NT * C::TILE;
  float2 *R = U + C::TILE;
  float2 *S = R + C::TILE;
  float2 *T = U;  // T replaces U after the r/s passes
  const int col = a + C::PJ * b;  // padded offset of the t-column (a, b, 0)
  double pw = 0.0;  // p.w of this thread's points (binary64 across elements)
  const int64_t estride = (int64_t)gridDim.x * C::ELB;
  // Range guard. Elements whose inputs lie in [2^-60, 2^61) (zeros aside)
  // are computed unscaled: every double-float value stays far inside the
  // binary32 exponent range. Any other element (rare: a thread saw a value
  // above 2^60, or only values below 2^-60) is redone at the power-of-two
  // scale 2^-sh of its largest input, so any finite input is accepted.
  // s_bad: some element of the CTA needs the scaled path (CTA-wide, so the
  // extra barriers of that path are uniform); s_emax: per element, its
  // largest binary64 exponent field.
  __shared__ int s_emax[C::ELB];
  __shared__ int s_bad;
  if (tid < C::ELB) s_emax[tid] = 0;
  if (tid == 0) s_bad = 0;
  __syncthreads();

  int32_t go[NP];  // gather indices of this thread's column, kept for the scatter
  float2 uk[NP];   // its (scaled) u values, kept for p.w and the Helmholtz term (T replaces the U tile)
  int sh = 0;      // the element's scale: values are carried as x 2^-sh
  for (int64_t e0 = (int64_t)blockIdx.x * C::ELB; e0 < E; e0 += estride) {
    const int64_t ei = e0 + le;  // position in the element list (or the element itself)
    const bool act = ei < E;
    const int64_t e = !act ? E : (elist ? (int64_t)elist[ei] : ei);  // inactive: never dereferenced
    // P0: gather and split the t-column; one thread per element starts the
    // L2 prefetch of the element's geometric factors (read in P2)
    if (act && t == 0) prefetch_l2(Gdf + e * 6 * C::N3, 48u * C::N3);
    // the mass term's B (read in P4) likewise; its block is 16-byte aligned
    // and a multiple of 16 bytes when NP^3 is even
    if constexpr (HELM && C::N3 % 2 == 0)
      if (act && t == 1) prefetch_l2(Bdf + e * C::N3, 8u * C::N3);
    {
      double v[NP];
      if (ASSEMBLED) {  // all indices, then all values: one round trip each
#pragma unroll
        for (int k = 0; k < NP; ++k) go[k] = act ? l2gm[e * C::N3 + a + NP * b + C::N2 * k] : -1;
#pragma unroll
        for (int k = 0; k < NP; ++k) v[k] = (go[k] >= 0) ? u[go[k]] : 0.0;
      } else {
#pragma unroll
        for (int k = 0; k < NP; ++k) v[k] = act ? u[e * C::N3 + a + NP * b + C::N2 * k] : 0.0;
      }
      int em = 0;
#pragma unroll
      for (int k = 0; k < NP; ++k) em = max(em, df::exp_field(v[k]));
      if (em > 1023 + 60 || (em != 0 && em < 1023 - 60)) s_bad = 1;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        uk[k] = df::from_f64(v[k]);
        U[col + C::PK * k] = uk[k];
      }
    }
    sh = 0;
    __syncthreads();
    if (s_bad) {  // rare, uniform over the CTA: redo P0 of the flagged CTA at the elements' scales
      int em = 0;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const double vk = ASSEMBLED ? ((go[k] >= 0) ? u[go[k]] : 0.0) : (act ? u[e * C::N3 + a + NP * b + C::N2 * k] : 0.0);
        em = max(em, df::exp_field(vk));
      }
      atomicMax(&s_emax[le], em);
      __syncthreads();
      sh = s_emax[le] - 1023;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const double vk = ASSEMBLED ? ((go[k] >= 0) ? u[go[k]] : 0.0) : (act ? u[e * C::N3 + a + NP * b + C::N2 * k] : 0.0);
        uk[k] = df::from_f64_scaled(vk, sh);
        U[col + C::PK * k] = uk[k];
      }
      __syncthreads();
    }
    // P1: forward contractions, r-, s- and t-lines, one loop body (T
    // replaces U: the t-lines wait until every thread has read its r/s lines)
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      if (d == 2) __syncthreads();
      const int base = d == 0 ? C::PJ * a + C::PK * b : (d == 1 ? a + C::PK * b : col);
      const int str = d == 0 ? 1 : (d == 1 ? C::PJ : C::PK);
      float2 *O = d == 0 ? R : (d == 1 ? S : T);
      float2 y[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) y[m] = U[base + str * m];
      if constexpr (NP % 2 == 0) {
        line_apply_store<NP, false>(y, O, base, str, kq);
      } else {
        float2 z[NP];
        line_apply<NP, false>(y, z);
#pragma unroll
        for (int m = 0; m < NP; ++m) O[base + str * m] = z[m];
      }
    }
    __syncthreads();
    if (tid == 0) s_bad = 0;  // every thread has read the flags and scales of this element group
    if (t == 0) s_emax[le] = 0;
    // P2: metric on the t-column (a, b, :), in place
    const float2 *Ge = Gdf + (act ? e : 0) * 6 * C::N3 + a + NP * b;
    float2 gn[6];  // level k + 1's factors, loaded while level k is computed
#pragma unroll
    for (int f = 0; f < 6; ++f) gn[f] = act ? Ge[f * C::N3] : make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int q = col + C::PK * k;
      const float2 ur = R[q], us = S[q], uu = T[q];
      float2 g[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) g[f] = gn[f];
      if (k + 1 < NP) {
#pragma unroll
        for (int f = 0; f < 6; ++f) gn[f] = act ? Ge[f * C::N3 + C::N2 * (k + 1)] : make_float2(0.0f, 0.0f);
      }
      R[q] = metric_row(g[0], g[1], g[2], ur, us, uu);
      S[q] = metric_row(g[1], g[3], g[4], ur, us, uu);
      T[q] = metric_row(g[2], g[4], g[5], ur, us, uu);
    }
    __syncthreads();
    // P3: transposed contractions in place (lines of one direction are disjoint)
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      const int base = d == 0 ? C::PJ * a + C::PK * b : (d == 1 ? a + C::PK * b : col);
      const int str = d == 0 ? 1 : (d == 1 ? C::PJ : C::PK);
      float2 *O = d == 0 ? R : (d == 1 ? S : T);
      float2 y[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) y[m] = O[base + str * m];
      if constexpr (NP % 2 == 0) {
        line_apply_store<NP, true>(y, O, base, str, kq);
      } else {
        float2 z[NP];
        line_apply<NP, true>(y, z);
#pragma unroll
        for (int m = 0; m < NP; ++m) O[base + str * m] = z[m];
      }
    }
    __syncthreads();
    // P4: sum the three directions, scale, convert, write
    df::Acc pwe = {0.0f, 0.0f};  // this element's p.w terms (scaled by 2^-2sh)
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int q = col + C::PK * k;
      const int p = a + NP * b + C::N2 * k;
      const float2 zr = R[q], zs = S[q], zt = T[q];
      df::Acc acc = {zt.x, zt.y};
      df::acc_add(acc, zr.x, zr.y);
      df::acc_add(acc, zs.x, zs.y);
      float2 v;
      df::fast_two_sum(acc.s, acc.c, v.x, v.y);
      if (HELM) {
        const float2 xk = uk[k];  // u at the point, from P0 (the U tile now holds T)
        const float2 Bv = act ? Bdf[e * C::N3 + p] : make_float2(0.0f, 0.0f);
        const float2 buv = df::norm(df::mul_first(Bv.x, Bv.y, xk.x, xk.y));
        df::Acc o = df::mul_first(h1.x, h1.y, v.x, v.y);
        df::mac(o, h2.x, h2.y, buv.x, buv.y);
        v = df::norm(o);
      }
      if (act) {
        const double vd = df::to_f64_scaled(v.x, v.y, sh);
        if (ASSEMBLED) {
          const int32_t g = go[k];
          if (wloc) wloc[e * C::N3 + p] = (g >= 0) ? vd : 0.0;
          else if (g >= 0) atomicAdd(&w[g], vd);
          if (pw_partial) {  // u at the point: the thread's own values from P0
            const float2 xk = uk[k];
            df::mac(pwe, xk.x, xk.y, v.x, v.y);
          }
        } else {
          w[e * C::N3 + p] = vd;
        }
      }
    }
    if (ASSEMBLED && pw_partial != nullptr) {
      const float2 pn = df::norm(pwe);
      pw += df::to_f64_scaled(pn.x, pn.y, 2 * sh);
    }
    __syncthreads();
  }
  if (ASSEMBLED && pw_partial != nullptr) {
    // fixed-order sums: a shuffle tree per warp, one partial per warp, when
    // the CTA is whole warps; else (a partial warp) a serial CTA sum over
    // shared memory
    double v = pw;
    if constexpr (C::THREADS % 32 == 0) {
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if ((tid & 31) == 0) pw_partial[(int64_t)blockIdx.x * C::PW_PARTS + (tid >> 5)] = v;
    } else {
      double *red = reinterpret_cast<double *>(sm2);  // the tiles are free after the last barrier
      red[tid] = v;
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int q = 0; q < C::THREADS; ++q) s += red[q];
        pw_partial[blockIdx.x] = s;
      }
    }
  }
}

// ---------------------------------------------------------------- field operators
// The same element-local machinery for the explicit terms of the time step
// (Sec. 2.2: derivatives carried to deformed elements by the chain rule).
// Rdf is the inverse Jacobian dr_a/dx_c at every point, split to (hi, lo),
// laid out [E][9][n3] with factor 3a + c.
template <int NP>
struct FieldCfg {
  using C = DfCfg<NP>;
  static constexpr int SMEM = 2 * C::TILE * C::ELB * (int)sizeof(float2);
};

// physical gradient of an E-vector: d_a = D_a f along the three element
// directions, then g_c = sum_a dr_a/dx_c d_a
template <int NP>
__global__ void __launch_bounds__(DfCfg<NP>::THREADS)
    k_grad_df64(int64_t E, const float2 *__restrict__ Rdf, const double *__restrict__ f, double *__restrict__ g0,
                double *__restrict__ g1, double *__restrict__ g2) {
  using C = DfCfg<NP>;
  extern __shared__ float2 sm2[];
  const int tid = threadIdx.x;
  const int le = tid / C::N2;
  const int t = tid - le * C::N2;
  const int a = t % NP, b = t / NP;
  float2 *Rt = sm2 + le * 2 * C::TILE;  // the field, then its r-derivative
  float2 *St = Rt + C::TILE;            // its s-derivative
  const int col = a + C::PJ * b;
  const int64_t estride = (int64_t)gridDim.x * C::ELB;
  for (int64_t e0 = (int64_t)blockIdx.x * C::ELB; e0 < E; e0 += estride) {
    const int64_t e = e0 + le;
    const bool act = e < E;
    float2 x[NP], zt[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      x[k] = df::from_f64(act ? f[e * C::N3 + a + NP * b + C::N2 * k] : 0.0);
      Rt[col + C::PK * k] = x[k];
    }
    __syncthreads();
    // s-lines first into St (reads the field in Rt), then the r-lines in place
    // after a barrier, and the t-line from registers
    {
      float2 y[NP], z[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) y[m] = Rt[a + C::PK * b + C::PJ * m];
      line_apply<NP, false>(y, z);
#pragma unroll
      for (int m = 0; m < NP; ++m) St[a + C::PK * b + C::PJ * m] = z[m];
#pragma unroll
      for (int m = 0; m < NP; ++m) y[m] = Rt[C::PJ * a + C::PK * b + m];
      __syncthreads();
      line_apply<NP, false>(y, z);
#pragma unroll
      for (int m = 0; m < NP; ++m) Rt[C::PJ * a + C::PK * b + m] = z[m];
    }
    line_apply<NP, false>(x, zt);
    __syncthreads();
    if (act) {
      const float2 *Re = Rdf + e * 9 * C::N3 + a + NP * b;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int q = col + C::PK * k;
        const int64_t p = e * C::N3 + a + NP * b + C::N2 * k;
        const float2 dr = Rt[q], ds = St[q], dtt = zt[k];
        float2 r[9];
#pragma unroll
        for (int f9 = 0; f9 < 9; ++f9) r[f9] = Re[f9 * C::N3 + C::N2 * k];
        float2 v = metric_row(r[0], r[3], r[6], dr, ds, dtt);
        g0[p] = df::to_f64(v.x, v.y);
        v = metric_row(r[1], r[4], r[7], dr, ds, dtt);
        g1[p] = df::to_f64(v.x, v.y);
        v = metric_row(r[2], r[5], r[8], dr, ds, dtt);
        g2[p] = df::to_f64(v.x, v.y);
      }
    }
    __syncthreads();
  }
}

// weak divergence of a vector E-field: out = sum_a D_a^T v_a with
// v_a = B sum_c dr_a/dx_c f_c
template <int NP>
__global__ void __launch_bounds__(DfCfg<NP>::THREADS)
    k_wdiv_df64(int64_t E, const float2 *__restrict__ Rdf, const float2 *__restrict__ Bdf,
                const double *__restrict__ f0, const double *__restrict__ f1, const double *__restrict__ f2,
                double *__restrict__ out) {
  using C = DfCfg<NP>;
  extern __shared__ float2 sm2[];
  const int tid = threadIdx.x;
  const int le = tid / C::N2;
  const int t = tid - le * C::N2;
  const int a = t % NP, b = t / NP;
  float2 *Rt = sm2 + le * 2 * C::TILE;
  float2 *St = Rt + C::TILE;
  const int col = a + C::PJ * b;
  const int64_t estride = (int64_t)gridDim.x * C::ELB;
  for (int64_t e0 = (int64_t)blockIdx.x * C::ELB; e0 < E; e0 += estride) {
    const int64_t e = e0 + le;
    const bool act = e < E;
    const int64_t ec = act ? e : 0;
    const float2 *Re = Rdf + ec * 9 * C::N3 + a + NP * b;
    float2 vt[NP], zt[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int64_t p = ec * C::N3 + a + NP * b + C::N2 * k;
      const float2 fa = df::from_f64(act ? f0[p] : 0.0), fb = df::from_f64(act ? f1[p] : 0.0),
                   fc = df::from_f64(act ? f2[p] : 0.0);
      const float2 bw = Bdf[p];
      float2 r[9];
#pragma unroll
      for (int f9 = 0; f9 < 9; ++f9) r[f9] = Re[f9 * C::N3 + C::N2 * k];
      float2 v = metric_row(r[0], r[1], r[2], fa, fb, fc);
      Rt[col + C::PK * k] = df::norm(df::mul_first(bw.x, bw.y, v.x, v.y));
      v = metric_row(r[3], r[4], r[5], fa, fb, fc);
      St[col + C::PK * k] = df::norm(df::mul_first(bw.x, bw.y, v.x, v.y));
      v = metric_row(r[6], r[7], r[8], fa, fb, fc);
      vt[k] = df::norm(df::mul_first(bw.x, bw.y, v.x, v.y));
    }
    __syncthreads();
    // transposed contractions in place (the lines of one direction are disjoint)
#pragma unroll 1
    for (int d = 0; d < 2; ++d) {
      const int base = d == 0 ? C::PJ * a + C::PK * b : a + C::PK * b;
      const int str = d == 0 ? 1 : C::PJ;
      float2 *O = d == 0 ? Rt : St;
      float2 y[NP], z[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) y[m] = O[base + str * m];
      line_apply<NP, true>(y, z);
#pragma unroll
      for (int m = 0; m < NP; ++m) O[base + str * m] = z[m];
    }
    line_apply<NP, true>(vt, zt);
    __syncthreads();
    if (act) {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int q = col + C::PK * k;
        const float2 zr = Rt[q], zs = St[q];
        df::Acc acc = {zt[k].x, zt[k].y};
        df::acc_add(acc, zr.x, zr.y);
        df::acc_add(acc, zs.x, zs.y);
        float2 v;
        df::fast_two_sum(acc.s, acc.c, v.x, v.y);
        out[e * C::N3 + a + NP * b + C::N2 * k] = df::to_f64(v.x, v.y);
      }
    }
    __syncthreads();
  }
}

__global__ void k_split_df64(int64_t n, const double *__restrict__ x, float2 *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = df::from_f64(x[i]);
}

template <int NP, bool GRAD>
int launch_field_np(const sem_mesh *m, const float2 *Rdf, const double *f0, const double *f1, const double *f2,
                    double *o0, double *o1, double *o2, cudaStream_t st) {
  using C = DfCfg<NP>;
  constexpr int smem = FieldCfg<NP>::SMEM;
  const unsigned grid = (unsigned)std::max<int64_t>((m->E + C::ELB - 1) / C::ELB, 1);
  if constexpr (GRAD) {
    auto kern = k_grad_df64<NP>;
    if (smem > 48 * 1024) SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    kern<<<grid, C::THREADS, smem, st>>>(m->E, Rdf, f0, o0, o1, o2);
    SEM_LAUNCH_CHECK("k_grad_df64");
  } else {
    auto kern = k_wdiv_df64<NP>;
    if (smem > 48 * 1024) SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    kern<<<grid, C::THREADS, smem, st>>>(m->E, Rdf, m->Bdf, f0, f1, f2, o0);
    SEM_LAUNCH_CHECK("k_wdiv_df64");
  }
  return SEM_OK;
}

template <bool GRAD>
int launch_field(const sem_mesh *m, const float2 *Rdf, const double *f0, const double *f1, const double *f2,
                 double *o0, double *o1, double *o2, cudaStream_t st) {
  if (int rc = ensure_tables(m->device)) return rc;
  switch (m->n) {
#define CASE(NPV) \
  case NPV:       \
    return launch_field_np<NPV, GRAD>(m, Rdf, f0, f1, f2, o0, o1, o2, st);
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
#undef CASE
    default:
      return sem_fail(SEM_ERR_INVALID_ARG, "unsupported polynomial order");
  }
}

// Grid of the operator: one CTA per element group (with p.w accumulation,
// PW_PARTS partial sums per CTA, so their number is a property of the mesh)
template <int NP>
int df_grid(const sem_mesh *m, unsigned *grid) {
  using C = DfCfg<NP>;
  *grid = (unsigned)std::max<int64_t>((m->E + C::ELB - 1) / C::ELB, 1);
  return SEM_OK;
}

template <int NP>
int launch_np(const sem_mesh *m, double h1, double h2, const double *u, double *w, double *pw_partial, bool assembled,
              cudaStream_t st, const int32_t *map, const int *skip, const int32_t *elist = nullptr,
              int64_t nlist = 0) {
  using C = DfCfg<NP>;
  unsigned grid;
  // one CTA per element group (the hardware scheduler balances the SMs; a
  // single resident wave of persistent CTAs measured 11 % slower)
  if (int rc = df_grid<NP>(m, &grid)) return rc;
  const int64_t nE = elist ? nlist : m->E;
  if (elist) grid = (unsigned)std::max<int64_t>((nlist + C::ELB - 1) / C::ELB, 1);
  const float2 h1d = split_host(h1), h2d = split_host(h2);
  const bool helm = !(h1 == 1.0 && h2 == 0.0);
  double *wloc = (assembled && !elist) ? (double *)m->det_w : nullptr;
#define LAUNCH(ASM, HLM)                                                                                  \
  do {                                                                                                    \
    auto kern = k_ax_df64<NP, ASM, HLM>;                                                                  \
    constexpr int smem = C::smem_ax(HLM);                                                                 \
    if (smem > 48 * 1024)                                                                                 \
      SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));           \
    kern<<<grid, C::THREADS, smem, st>>>(nE, m->Gdf, m->Bdf, h1d, h2d, u, w, map, pw_partial, wloc, skip, \
                                         elist);                                                          \
  } while (0)
  if (assembled) {
    if (helm) LAUNCH(true, true);
    else LAUNCH(true, false);
  } else {
    if (helm) LAUNCH(false, true);
    else LAUNCH(false, false);
  }
#undef LAUNCH
  SEM_LAUNCH_CHECK("k_ax_df64");
  if (wloc) return sem_launch_gather_add(m, wloc, w, st);
  return SEM_OK;
}

}  // namespace

int sem_df64_pw_count(const sem_mesh *m) {
  unsigned grid = 0;
  int rc = SEM_OK;
  switch (m->n) {
#define CASE(NPV)                              \
  case NPV:                                    \
    rc = df_grid<NPV>(m, &grid);               \
    grid *= DfCfg<NPV>::PW_PARTS;              \
    break;
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
#undef CASE
    default:
      return 0;
  }
  return rc == SEM_OK ? (int)grid : 0;
}

int sem_launch_ax_df64(const sem_mesh *m, double h1, double h2, const double *u, double *w, double *pw_partial,
                       bool assembled, cudaStream_t st, const int32_t *map, const int *skip) {
  if (m->n == 8 && m->use_tc == 1) return sem_launch_ax_tc(m, h1, h2, u, w, pw_partial, assembled, st, map, skip);
  if (m->n == 8 && m->use_tc == 2 && m->Gt && h1 == 1.0 && h2 == 0.0 && (!assembled || map == m->l2gm))
    return sem_launch_ax_tcr(m, u, w, pw_partial, assembled, st, skip);
  if (int rc = ensure_tables(m->device)) return rc;
  switch (m->n) {
#define CASE(NPV) \
  case NPV:       \
    return launch_np<NPV>(m, h1, h2, u, w, pw_partial, assembled, st, map, skip);
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
#undef CASE
    default:
      return sem_fail(SEM_ERR_INVALID_ARG, "unsupported polynomial order");
  }
}

int sem_launch_ax_df64_list(const sem_mesh *m, double h1, double h2, const double *u, double *w, cudaStream_t st,
                            const int32_t *elist, int64_t nlist) {
  if (m->n == 8 && m->use_tc == 1)
    return sem_launch_ax_tc(m, h1, h2, u, w, nullptr, true, st, m->l2gm, nullptr, elist, nlist);
  if (int rc = ensure_tables(m->device)) return rc;
  switch (m->n) {
#define CASE(NPV) \
  case NPV:       \
    return launch_np<NPV>(m, h1, h2, u, w, nullptr, true, st, m->l2gm, nullptr, elist, nlist);
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
#undef CASE
    default:
      return sem_fail(SEM_ERR_INVALID_ARG, "unsupported polynomial order");
  }
}

int sem_launch_grad_df64(const sem_mesh *m, const float2 *Rdf, const double *f, double *g0, double *g1, double *g2,
                         cudaStream_t st) {
  return launch_field<true>(m, Rdf, f, nullptr, nullptr, g0, g1, g2, st);
}

int sem_launch_wdiv_df64(const sem_mesh *m, const float2 *Rdf, const double *f0, const double *f1, const double *f2,
                         double *out, cudaStream_t st) {
  return launch_field<false>(m, Rdf, f0, f1, f2, out, nullptr, nullptr, st);
}

int sem_launch_split_df64(const double *x, float2 *y, int64_t n, cudaStream_t st) {
  if (n <= 0) return SEM_OK;
  k_split_df64<<<grid_for(n, 256), 256, 0, st>>>(n, x, y);
  SEM_LAUNCH_CHECK("k_split_df64");
  return SEM_OK;
}
