// binary64-accurate matrix-free Helmholtz operator in double-float
// arithmetic on the binary32 pipe (same operator as sem_ax.cu, Sec. 2.2).
//
// Why: on GB300 binary64 FMA runs at ~1.2 TFLOP/s against ~74 TFLOP/s for
// binary32, so the native-FP64 operator is bound by the FP64 pipe at about
// ten times the HBM time. Carrying every value as hi + lo binary32 with
// error-free transformations costs ~10 binary32 operations per binary64
// multiply-add and keeps ~2^-46 relative accuracy.
//
// Structure per element (NP = N+1 points per direction, NP^2 threads):
//   P0  gather u (binary64), split to df64; thread (a,b) keeps the t-line
//       u(a,b,:) in registers and stores it to the shared tile U
//   P1  each thread contracts three lines with D: its t-line (registers),
//       the r-line u(:,a,b) and the s-line u(a,:,b) (shared tile) -> R, S
//   P2  pointwise metric on its t-column: (wr, ws, wt) = G (ur, us, ut)
//   P3  transposed contractions: r-lines of R and s-lines of S in place,
//       the t-line in registers
//   P4  w(a,b,:) = t-part + R + S, then h1 w + h2 B u, back to binary64
// The 1-D contractions use the even-odd split of the centro-antisymmetric
// D (D[N-i][N-j] = -D[i][j]), which halves the multiply-adds.
#include <algorithm>
#include <mutex>
#include <vector>

#include "sem_df64.cuh"
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

// y = M x along one line (M = D, or D^T when TR), df64 in, normalised df64 out
template <int NP, bool TR>
__device__ __forceinline__ void line_apply(const float2 (&x)[NP], float2 (&y)[NP]) {
  constexpr int N = NP - 1;
  if constexpr (NP % 2 == 0) {
    constexpr int H = NP / 2;
    const float2 *A = c_tab + tab_off(NP) + (TR ? 2 * H * H : 0);
    const float2 *Bq = A + H * H;
    df::Acc xe[H], xo[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
      df::two_sum(x[m].x, x[N - m].x, xe[m].s, xe[m].c);
      xe[m].c = df::add(xe[m].c, df::add(x[m].y, x[N - m].y));
      df::two_sum(x[m].x, -x[N - m].x, xo[m].s, xo[m].c);
      xo[m].c = df::add(xo[m].c, df::sub(x[m].y, x[N - m].y));
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
      df::Acc P = df::mul_first(A[i * H].x, A[i * H].y, xe[0].s, xe[0].c);
      df::Acc Q = df::mul_first(Bq[i * H].x, Bq[i * H].y, xo[0].s, xo[0].c);
#pragma unroll
      for (int m = 1; m < H; ++m) {
        df::mac(P, A[i * H + m].x, A[i * H + m].y, xe[m].s, xe[m].c);
        df::mac(Q, Bq[i * H + m].x, Bq[i * H + m].y, xo[m].s, xo[m].c);
      }
      y[i] = df::norm(df::sum(P, Q));
      y[N - i] = df::norm(df::diff(Q, P));
    }
  } else {
    const float2 *M = c_tab + tab_off(NP) + (TR ? NP * NP : 0);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      df::Acc a = df::mul_first(M[i * NP].x, M[i * NP].y, x[0].x, x[0].y);
#pragma unroll
      for (int m = 1; m < NP; ++m) df::mac(a, M[i * NP + m].x, M[i * NP + m].y, x[m].x, x[m].y);
      y[i] = df::norm(a);
    }
  }
}

template <int NP>
struct DfCfg {
  static constexpr int N2 = NP * NP;
  static constexpr int N3 = NP * NP * NP;
  static constexpr int PJ = NP + 1;        // padded r-line stride (avoids bank conflicts)
  static constexpr int PK = NP * (NP + 1);
  static constexpr int TILE = NP * PK;     // float2 per tile
  static constexpr int ELB = (N2 >= 128) ? 1 : (128 / N2 > 4 ? 4 : 128 / N2);
  static constexpr int THREADS = N2 * ELB;
  static constexpr int SMEM = 3 * TILE * ELB * (int)sizeof(float2);
};

template <int NP, bool ASSEMBLED, bool HELM>
__global__ void __launch_bounds__(DfCfg<NP>::THREADS)
    k_ax_df64(int64_t E, const float2 *__restrict__ Gdf, const float2 *__restrict__ Bdf, float2 h1, float2 h2,
              const double *__restrict__ u, double *__restrict__ w, const int32_t *__restrict__ l2gm,
              double *__restrict__ pw_partial) {
  using C = DfCfg<NP>;
  extern __shared__ float2 sm2[];
  const int tid = threadIdx.x;
  const int le = tid / C::N2;
  const int t = tid - le * C::N2;
  const int a = t % NP, b = t / NP;
  float2 *U = sm2 + le * 3 * C::TILE;
  float2 *R = U + C::TILE;
  float2 *S = R + C::TILE;
  auto P = [](int i, int j, int k) { return i + C::PJ * j + C::PK * k; };
  df::Acc pw = {0.0f, 0.0f};

  for (int64_t e0 = (int64_t)blockIdx.x * C::ELB; e0 < E; e0 += (int64_t)gridDim.x * C::ELB) {
    const int64_t e = e0 + le;
    const bool act = e < E;
    // P0: gather and split
    float2 x[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = a + NP * b + C::N2 * k;
      double v = 0.0;
      if (act) {
        if (ASSEMBLED) {
          const int32_t g = l2gm[e * C::N3 + p];
          v = (g >= 0) ? u[g] : 0.0;
        } else {
          v = u[e * C::N3 + p];
        }
      }
      x[k] = df::from_f64(v);
      U[P(a, b, k)] = x[k];
    }
    __syncthreads();
    // P1: forward contractions
    float2 ut[NP];
    line_apply<NP, false>(x, ut);
    {
      float2 y[NP], z[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) y[m] = U[P(m, a, b)];
      line_apply<NP, false>(y, z);
#pragma unroll
      for (int m = 0; m < NP; ++m) R[P(m, a, b)] = z[m];
#pragma unroll
      for (int m = 0; m < NP; ++m) y[m] = U[P(a, m, b)];
      line_apply<NP, false>(y, z);
#pragma unroll
      for (int m = 0; m < NP; ++m) S[P(a, m, b)] = z[m];
    }
    __syncthreads();
    // P2: metric on the t-column (a, b, :)
    float2 wt[NP];
    const float2 *Ge = Gdf + (act ? e : 0) * 6 * C::N3;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = a + NP * b + C::N2 * k;
      const float2 ur = R[P(a, b, k)], us = S[P(a, b, k)], uu = ut[k];
      float2 g[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) g[f] = act ? Ge[f * C::N3 + p] : make_float2(0.0f, 0.0f);
      df::Acc r = df::mul_first(g[0].x, g[0].y, ur.x, ur.y);
      df::mac(r, g[1].x, g[1].y, us.x, us.y);
      df::mac(r, g[2].x, g[2].y, uu.x, uu.y);
      df::Acc s = df::mul_first(g[1].x, g[1].y, ur.x, ur.y);
      df::mac(s, g[3].x, g[3].y, us.x, us.y);
      df::mac(s, g[4].x, g[4].y, uu.x, uu.y);
      df::Acc q = df::mul_first(g[2].x, g[2].y, ur.x, ur.y);
      df::mac(q, g[4].x, g[4].y, us.x, us.y);
      df::mac(q, g[5].x, g[5].y, uu.x, uu.y);
      R[P(a, b, k)] = df::norm(r);
      S[P(a, b, k)] = df::norm(s);
      wt[k] = df::norm(q);
    }
    __syncthreads();
    // P3: transposed contractions (r- and s-lines in place)
    float2 zt[NP];
    line_apply<NP, true>(wt, zt);
    {
      float2 y[NP], z[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) y[m] = R[P(m, a, b)];
      line_apply<NP, true>(y, z);
#pragma unroll
      for (int m = 0; m < NP; ++m) R[P(m, a, b)] = z[m];
#pragma unroll
      for (int m = 0; m < NP; ++m) y[m] = S[P(a, m, b)];
      line_apply<NP, true>(y, z);
#pragma unroll
      for (int m = 0; m < NP; ++m) S[P(a, m, b)] = z[m];
    }
    __syncthreads();
    // P4: sum the three directions, scale, convert, write
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = a + NP * b + C::N2 * k;
      const float2 zr = R[P(a, b, k)], zs = S[P(a, b, k)];
      df::Acc acc = {zt[k].x, zt[k].y};
      df::acc_add(acc, zr.x, zr.y);
      df::acc_add(acc, zs.x, zs.y);
      float2 v = df::norm(acc);
      if (HELM) {
        const float2 Bv = act ? Bdf[e * C::N3 + p] : make_float2(0.0f, 0.0f);
        df::Acc bu = df::mul_first(Bv.x, Bv.y, x[k].x, x[k].y);
        const float2 buv = df::norm(bu);
        df::Acc o = df::mul_first(h1.x, h1.y, v.x, v.y);
        df::mac(o, h2.x, h2.y, buv.x, buv.y);
        v = df::norm(o);
      }
      if (act) {
        const double vd = df::to_f64(v.x, v.y);
        if (ASSEMBLED) {
          const int32_t g = l2gm[e * C::N3 + p];
          if (g >= 0) atomicAdd(&w[g], vd);
          if (pw_partial) df::mac(pw, x[k].x, x[k].y, v.x, v.y);
        } else {
          w[e * C::N3 + p] = vd;
        }
      }
    }
    __syncthreads();
  }
  if (ASSEMBLED && pw_partial != nullptr) {
    __shared__ double red[32];
    const float2 pn = df::norm(pw);
    double v = (double)pn.x + (double)pn.y;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int q = 0; q < (C::THREADS + 31) / 32; ++q) s += red[q];
      pw_partial[blockIdx.x] = s;
    }
  }
}

template <int NP>
int launch_np(const sem_mesh *m, double h1, double h2, const double *u, double *w, double *pw_partial, bool assembled,
              cudaStream_t st) {
  using C = DfCfg<NP>;
  int64_t blocks = (m->E + C::ELB - 1) / C::ELB;
  if (assembled) blocks = std::min<int64_t>(blocks, 152 * 16);
  const unsigned grid = (unsigned)std::max<int64_t>(blocks, 1);
  const float2 h1d = split_host(h1), h2d = split_host(h2);
  const bool helm = !(h1 == 1.0 && h2 == 0.0);
#define LAUNCH(ASM, HLM)                                                                                    \
  do {                                                                                                      \
    auto kern = k_ax_df64<NP, ASM, HLM>;                                                                    \
    if (C::SMEM > 48 * 1024)                                                                                \
      SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));          \
    kern<<<grid, C::THREADS, C::SMEM, st>>>(m->E, m->Gdf, m->Bdf, h1d, h2d, u, w, m->l2gm, pw_partial);     \
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
  return SEM_OK;
}

}  // namespace

int sem_df64_grid(const sem_mesh *m) {
  // must match launch_np's assembled grid for every NP (used for partial sums)
  int elb;
  switch (m->n) {
#define CASE(NPV)                 \
  case NPV:                       \
    elb = DfCfg<NPV>::ELB;        \
    break;
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
#undef CASE
    default:
      return 0;
  }
  int64_t blocks = std::min<int64_t>((m->E + elb - 1) / elb, 152 * 16);
  return (int)std::max<int64_t>(blocks, 1);
}

int sem_launch_ax_df64(const sem_mesh *m, double h1, double h2, const double *u, double *w, double *pw_partial,
                       bool assembled, cudaStream_t st) {
  if (int rc = ensure_tables(m->device)) return rc;
  switch (m->n) {
#define CASE(NPV) \
  case NPV:       \
    return launch_np<NPV>(m, h1, h2, u, w, pw_partial, assembled, st);
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
#undef CASE
    default:
      return sem_fail(SEM_ERR_INVALID_ARG, "unsupported polynomial order");
  }
}
