// p-multigrid preconditioned flexible CG (Sec. 2.2: NekRS preconditions the
// pressure Poisson solve with p-multigrid and 4th-kind Chebyshev-accelerated
// smoothers, running most preconditioner work in FP32 to save bandwidth).
//
// Levels: the same elements at decreasing orders, each with its own mesh
// (geometry re-evaluated at the level's GLL points). Smoothing levels run in
// binary32 with geometric factors in binary32 or bfloat16; the coarsest level
// is a binary64-accurate (double-float operator) Jacobi-PCG solve. Transfer operators: element-wise
// tensor-product Lagrange interpolation P (coarse -> fine) and R = P^T.
// Smoother: 4th-kind Chebyshev in D^{-1}A (Lottes 2022 recurrence):
//   d_0 = 4/(3 lam) D^{-1} r_0;  for i = 1..k: x += d_{i-1}; (i < k) r -= A d_{i-1};
//   d_i = (2i-1)/(2i+3) d_{i-1} + (8i+4)/((2i+3) lam) D^{-1} r_i.
// Outer: flexible CG, beta = r.(z_new - z_old) / r.z_old.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "sem_df64.cuh"
#include "sem_internal.h"
#include "sem_tma.cuh"

namespace {

struct PmgLevel {
  sem_mesh *m = nullptr;
  bool own = false;
  const int32_t *map = nullptr;  // l2gm (Dirichlet mask) or l2g (pure Neumann)
  float *Gf = nullptr;
  __nv_bfloat16 *Gb = nullptr;
  float *Bf = nullptr;
  float *Df = nullptr;
  float *dinv = nullptr;
  float *minv = nullptr;  // 1 / multiplicity
  float lam = 0.0f;
  float *b = nullptr, *x = nullptr, *r = nullptr, *d = nullptr, *t = nullptr;
  int *err = nullptr;  // set by a kernel whose shared-memory copies did not land (then the persistent
                       // TMA operator is used; NULL selects the plain operator)
  // bfloat16 smoothing at N = 7: lane-major geometry, map and (Helmholtz)
  // mass of the tensor-core operator (sem_ax_bf16.cu); NULL otherwise
  void *Gl = nullptr, *Ml = nullptr, *Bl = nullptr;
  // binary64-accurate smoothing (SEM_PREC_DF64): the level's vectors in
  // binary64 and the double-float operator
  double *b64 = nullptr, *x64 = nullptr, *r64 = nullptr, *d64 = nullptr, *t64 = nullptr, *dinv64 = nullptr;
  double *minv64 = nullptr;
  double lam64 = 0.0;
};

constexpr int kPart = 152 * 2;

}  // namespace

struct sem_pmg {
  std::vector<PmgLevel> L;
  float *J[3] = {};  // device interpolation matrices, level l+1 -> l, [n_f][n_c]
  double *J64[3] = {};  // the same in binary64 (binary64-accurate smoothing)
  sem_pmg_opts o;
  double h1 = 1.0, h2 = 0.0;
  double *cb = nullptr, *cx = nullptr;  // coarsest level (binary64)
  double *cdinv = nullptr;              // its Jacobi inverse (persistent coarse solver)
  void *cws = nullptr;
  double *r = nullptr, *z = nullptr, *zn = nullptr, *p = nullptr, *w = nullptr;  // outer FCG
  double *part = nullptr, *pw_part = nullptr;
  int *err = nullptr;  // device flag of the persistent operator (a bulk copy that never landed)
  std::vector<void *> owned;
};

namespace {

// ---------------------------------------------------------------- binary32 operator
template <int NP>
struct F32Cfg {
  static constexpr int N2 = NP * NP;
  static constexpr int N3 = NP * NP * NP;
  static constexpr int ELB = (N2 >= 256) ? 1 : (256 / N2);
  static constexpr int THREADS = N2 * ELB;
  static constexpr int SMEM = (NP * (NP + 1) + 4 * N3 * ELB) * (int)sizeof(float);
  static constexpr int MINB = (NP <= 8) ? 4 : 2;  // resident CTAs per SM the registers must allow
};

__device__ __forceinline__ float ldg_real(const float *p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ldg_real(const __nv_bfloat16 *p, int64_t i) { return __bfloat162float(p[i]); }
// plain (generic) loads, for values staged in shared memory
__device__ __forceinline__ float lds_real(const float *p, int i) { return p[i]; }
__device__ __forceinline__ float lds_real(const __nv_bfloat16 *p, int i) { return __bfloat162float(p[i]); }

// w[g] += h1 (A u)[g] + h2 (B u)[g] through map (-1 = skip), binary32. The
// kernel is bound by memory: the u column and the t-direction flux stay in
// shared memory (not registers) so that four CTAs fit per SM, and the gather
// indices of the next element are prefetched.
template <int NP, typename GT>
__global__ void __launch_bounds__(F32Cfg<NP>::THREADS, F32Cfg<NP>::MINB)
    k_ax32(int64_t E, const float *__restrict__ Df, const GT *__restrict__ G, const float *__restrict__ B, float h1,
           float h2, const float *__restrict__ u, float *__restrict__ w, const int32_t *__restrict__ map,
           float *__restrict__ wloc) {
  using C = F32Cfg<NP>;
  extern __shared__ float smf[];
  float *sD = smf;
  const int tid = threadIdx.x;
  const int le = tid / C::N2;
  const int ij = tid - le * C::N2;
  const int i = ij % NP, j = ij / NP;
  float *s_u = smf + NP * (NP + 1) + le * 4 * C::N3;
  float *s_r = s_u + C::N3;
  float *s_s = s_r + C::N3;
  float *s_t = s_s + C::N3;
  for (int t = tid; t < NP * NP; t += C::THREADS) sD[(t / NP) * (NP + 1) + (t % NP)] = Df[t];
  const int64_t estride = (int64_t)gridDim.x * C::ELB;
  int32_t gi[NP];
  {
    const int64_t e = (int64_t)blockIdx.x * C::ELB + le;
#pragma unroll
    for (int k = 0; k < NP; ++k) gi[k] = (e < E) ? map[e * C::N3 + i + NP * j + C::N2 * k] : -1;
  }
  __syncthreads();
  for (int64_t e0 = (int64_t)blockIdx.x * C::ELB; e0 < E; e0 += estride) {
    const int64_t e = e0 + le;
    const bool act = e < E;
    int32_t go[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      go[k] = gi[k];
      s_u[i + NP * j + C::N2 * k] = (gi[k] >= 0) ? u[gi[k]] : 0.0f;
    }
    {
      const int64_t en = e + estride;
#pragma unroll
      for (int k = 0; k < NP; ++k) gi[k] = (en < E) ? map[en * C::N3 + i + NP * j + C::N2 * k] : -1;
    }
    __syncthreads();
    const int64_t gbase = (act ? e : 0) * 6 * C::N3;
#pragma unroll 2
    for (int k = 0; k < NP; ++k) {
      const int p = i + NP * j + C::N2 * k;
      float g00 = 0, g01 = 0, g02 = 0, g11 = 0, g12 = 0, g22 = 0;
      if (act) {
        g00 = ldg_real(G, gbase + p);
        g01 = ldg_real(G, gbase + C::N3 + p);
        g02 = ldg_real(G, gbase + 2 * C::N3 + p);
        g11 = ldg_real(G, gbase + 3 * C::N3 + p);
        g12 = ldg_real(G, gbase + 4 * C::N3 + p);
        g22 = ldg_real(G, gbase + 5 * C::N3 + p);
      }
      float ur = 0.0f, us = 0.0f, ut = 0.0f;
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        ur = fmaf(sD[i * (NP + 1) + m], s_u[m + NP * j + C::N2 * k], ur);
        us = fmaf(sD[j * (NP + 1) + m], s_u[i + NP * m + C::N2 * k], us);
        ut = fmaf(sD[k * (NP + 1) + m], s_u[i + NP * j + C::N2 * m], ut);
      }
      s_r[p] = g00 * ur + g01 * us + g02 * ut;
      s_s[p] = g01 * ur + g11 * us + g12 * ut;
      s_t[p] = g02 * ur + g12 * us + g22 * ut;
    }
    __syncthreads();
#pragma unroll 2
    for (int k = 0; k < NP; ++k) {
      const int p = i + NP * j + C::N2 * k;
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        acc = fmaf(sD[m * (NP + 1) + i], s_r[m + NP * j + C::N2 * k], acc);
        acc = fmaf(sD[m * (NP + 1) + j], s_s[i + NP * m + C::N2 * k], acc);
        acc = fmaf(sD[m * (NP + 1) + k], s_t[i + NP * j + C::N2 * m], acc);
      }
      float val = h1 * acc;
      if (h2 != 0.0f && act) val = fmaf(h2 * B[e * C::N3 + p], s_u[p], val);
      if (wloc) {
        if (act) wloc[e * C::N3 + p] = (go[k] >= 0) ? val : 0.0f;
      } else if (go[k] >= 0) {
        atomicAdd(&w[go[k]], val);
      }
    }
    __syncthreads();
  }
}

// Persistent form for even NP: each CTA walks element groups with a stride of
// the grid, as a three-stage pipeline. The group's geometric factors and
// gather indices (contiguous per element) come into shared memory by bulk
// asynchronous copies (TMA) two groups ahead, in a ring of three buffers with
// one mbarrier each; the gathered u values of the next group are copied into
// shared memory by per-thread asynchronous copies one group ahead. Neither the
// geometry stream nor the gather latency is then exposed to the arithmetic.
// Each thread keeps its rows of D and D^T in registers, takes the t-direction
// coefficients from constant memory (compile-time indices) and keeps its
// t-column of u and of the t-flux in registers; r-lines are read with vector
// loads. Dynamic shared memory: barriers | G[3][ELB][6][N3] |
// map[3][ELB][N3] | u[2][ELB][N3] | r, s fluxes [ELB][2][N3].
template <int NP, typename GT>
struct TmaCfg {
  static constexpr int N2 = NP * NP;
  static constexpr int N3 = NP * NP * NP;
  static constexpr int ELB = (N2 >= 64) ? 1 : 64 / N2;
  static constexpr int THREADS = N2 * ELB;
  static constexpr int STAGES = 3;
  static constexpr int GELEM = 6 * N3 * (int)sizeof(GT);  // bytes of G per element
  static constexpr int MELEM = N3 * 4;                     // bytes of map per element
  static constexpr int OFF_G = 128;
  static constexpr int OFF_M = OFF_G + STAGES * ELB * GELEM;
  static constexpr int OFF_U = OFF_M + STAGES * ELB * MELEM;
  static constexpr int OFF_T = OFF_U + 2 * ELB * N3 * 4;
  static constexpr int SMEM = OFF_T + 2 * ELB * N3 * 4;
  static_assert(GELEM % 16 == 0 && MELEM % 16 == 0, "bulk copies need 16-byte multiples");
};

// binary32 derivative matrices D (row-major) for NP = 2 .. SEM_MAXNP in
// constant memory: with compile-time indices they are instruction operands
__host__ __device__ constexpr int d32_off(int np) { return np <= 2 ? 0 : d32_off(np - 1) + (np - 1) * (np - 1); }
__constant__ float c_D32[d32_off(SEM_MAXNP + 1)];
std::mutex g_d32_mu;
unsigned g_d32_ready = 0;  // bit per device

int ensure_d32(int device) {
  std::lock_guard<std::mutex> lk(g_d32_mu);
  if (device < 32 && (g_d32_ready >> device) & 1u) return SEM_OK;
  std::vector<float> tab(d32_off(SEM_MAXNP + 1));
  for (int np = 2; np <= SEM_MAXNP; ++np) {
    double xi[SEM_MAXNP], rho[SEM_MAXNP], D[SEM_MAXNP * SEM_MAXNP];
    if (int rc = sem_gll_host(np - 1, xi, rho, D)) return rc;
    for (int t = 0; t < np * np; ++t) tab[d32_off(np) + t] = (float)D[t];
  }
  SEM_CUDA(cudaMemcpyToSymbol(c_D32, tab.data(), sizeof(float) * tab.size()));
  if (device < 32) g_d32_ready |= 1u << device;
  return SEM_OK;
}

// a contiguous line of NP floats from shared memory (vector loads; NP even)
template <int NP>
__device__ __forceinline__ void load_line(const float *p, float (&v)[NP]) {
  if constexpr (NP % 4 == 0) {
#pragma unroll
    for (int q = 0; q < NP / 4; ++q) {
      const float4 t = reinterpret_cast<const float4 *>(p)[q];
      v[4 * q] = t.x;
      v[4 * q + 1] = t.y;
      v[4 * q + 2] = t.z;
      v[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NP / 2; ++q) {
      const float2 t = reinterpret_cast<const float2 *>(p)[q];
      v[2 * q] = t.x;
      v[2 * q + 1] = t.y;
    }
  }
}

// 4-byte asynchronous global -> shared copy, zero-filled when !valid
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid) {
  const unsigned sa = tma::smem_u32(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int NP, typename GT>
__global__ void __launch_bounds__(TmaCfg<NP, GT>::THREADS)
    k_ax32_tma(int64_t E, const float *__restrict__ Df, const GT *__restrict__ G, const float *__restrict__ B,
               float h1, float h2, const float *__restrict__ u, float *__restrict__ w,
               const int32_t *__restrict__ map, float *__restrict__ wloc, int *__restrict__ err) {
  using C = TmaCfg<NP, GT>;
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smraw);
  GT *Gs = reinterpret_cast<GT *>(smraw + C::OFF_G);
  int32_t *Ms = reinterpret_cast<int32_t *>(smraw + C::OFF_M);
  float *Us = reinterpret_cast<float *>(smraw + C::OFF_U);
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  const int le = tid / C::N2;
  const int ij = tid - le * C::N2;
  const int i = ij % NP, j = ij / NP;
  float *s_r = reinterpret_cast<float *>(smraw + C::OFF_T) + le * 2 * C::N3;
  float *s_s = s_r + C::N3;
  const float *cD = c_D32 + d32_off(NP);
  float Dr[NP], Ds[NP], DrT[NP], DsT[NP];  // D[i][m], D[j][m], D[m][i], D[m][j]
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    Dr[m] = cD[i * NP + m];
    Ds[m] = cD[j * NP + m];
    DrT[m] = cD[m * NP + i];
    DsT[m] = cD[m * NP + j];
  }
  const int64_t ngroups = (E + C::ELB - 1) / C::ELB;
  const int64_t gstride = gridDim.x;
  if (tid == 0) {
    for (int b = 0; b < C::STAGES; ++b) tma::mbar_init(&bar[b], 1);
    tma::fence_mbar_init();
    abort_flag = 0;
  }
  __syncthreads();
  // thread 0: group g into ring slot b
  auto issue = [&](int64_t g, int b) {
    const int64_t e0 = g * C::ELB;
    const unsigned ne = (unsigned)((E - e0) < C::ELB ? (E - e0) : C::ELB);
    tma::mbar_arrive_expect_tx(&bar[b], ne * (unsigned)(C::GELEM + C::MELEM));
    tma::bulk_g2s(Gs + (size_t)b * C::ELB * 6 * C::N3, G + e0 * 6 * C::N3, ne * C::GELEM, &bar[b]);
    tma::bulk_g2s(Ms + (size_t)b * C::ELB * C::N3, map + e0 * C::N3, ne * C::MELEM, &bar[b]);
  };
  // every thread: asynchronous gather of its column of group g (map in slot b) into u buffer ub
  auto gather = [&](int64_t g, int b, int ub, bool ok) {
    const int64_t e = g * C::ELB + le;
    const bool act = ok && e < E;
    const int32_t *Me = Ms + (size_t)b * C::ELB * C::N3 + le * C::N3;
    float *Ue = Us + (size_t)ub * C::ELB * C::N3 + le * C::N3;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = ij + C::N2 * k;
      const int32_t gk = act ? Me[p] : -1;
      cp_async4(Ue + p, gk >= 0 ? u + gk : u, gk >= 0);
    }
  };
  // the wait for group number q (q-th group of this CTA) uses slot q % 3, phase (q / 3) & 1
  auto wait_group = [&](int q) { return tma::mbar_wait(&bar[q % 3], (unsigned)(q / 3) & 1u, tma::kWaitLimit); };

  const int64_t g0 = blockIdx.x;
  int issued = 0;  // groups issued so far (thread 0's count; the same on every thread by construction)
  if (tid == 0) {
    if (g0 < ngroups) issue(g0, 0);
    if (g0 + gstride < ngroups) issue(g0 + gstride, 1);
  }
  issued = (g0 < ngroups) + (g0 + gstride < ngroups);
  if (g0 < ngroups) {
    const bool ok = wait_group(0);
    if (!ok) abort_flag = 1;
    gather(g0, 0, 0, ok);
  }
  cp_async_commit();
  int q = 0;
  for (int64_t g = g0; g < ngroups; g += gstride, ++q) {
    const int b = q % 3;
    const int64_t gn = g + gstride, gnn = g + 2 * gstride;
    if (gnn < ngroups) {  // slot (q + 2) % 3 was released by the previous iteration's final barrier
      if (tid == 0) {
        tma::fence_proxy_async();
        issue(gnn, (q + 2) % 3);
      }
      ++issued;
    }
    if (gn < ngroups) {
      const bool ok = wait_group(q + 1);
      if (!ok) abort_flag = 1;
      gather(gn, (q + 1) % 3, (q + 1) & 1, ok);
    }
    cp_async_commit();
    cp_async_wait_prev();  // this thread's gathers of group g have landed
    __syncthreads();
    if (abort_flag) break;
    const int64_t e = g * C::ELB + le;
    const GT *Ge = Gs + (size_t)b * C::ELB * 6 * C::N3 + le * 6 * C::N3;
    const int32_t *Me = Ms + (size_t)b * C::ELB * C::N3 + le * C::N3;
    const float *s_u = Us + (size_t)(q & 1) * C::ELB * C::N3 + le * C::N3;
    float ucol[NP], tt[NP];  // this thread's t-column of u, then of the t-flux
#pragma unroll
    for (int m = 0; m < NP; ++m) ucol[m] = s_u[ij + C::N2 * m];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = ij + C::N2 * k;
      const float g00 = lds_real(Ge, p), g01 = lds_real(Ge, C::N3 + p), g02 = lds_real(Ge, 2 * C::N3 + p),
                  g11 = lds_real(Ge, 3 * C::N3 + p), g12 = lds_real(Ge, 4 * C::N3 + p),
                  g22 = lds_real(Ge, 5 * C::N3 + p);
      float rl[NP];
      load_line<NP>(s_u + NP * j + C::N2 * k, rl);
      float ur = 0.0f, us = 0.0f, ut = 0.0f;
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        ur = fmaf(Dr[m], rl[m], ur);
        us = fmaf(Ds[m], s_u[i + NP * m + C::N2 * k], us);
        ut = fmaf(cD[k * NP + m], ucol[m], ut);
      }
      s_r[p] = g00 * ur + g01 * us + g02 * ut;
      s_s[p] = g01 * ur + g11 * us + g12 * ut;
      tt[k] = g02 * ur + g12 * us + g22 * ut;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = ij + C::N2 * k;
      float rl[NP];
      load_line<NP>(s_r + NP * j + C::N2 * k, rl);
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        acc = fmaf(DrT[m], rl[m], acc);
        acc = fmaf(DsT[m], s_s[i + NP * m + C::N2 * k], acc);
        acc = fmaf(cD[m * NP + k], tt[m], acc);
      }
      float val = h1 * acc;
      if (h2 != 0.0f && e < E) val = fmaf(h2 * B[e * C::N3 + p], s_u[p], val);
      const int32_t gk = (e < E) ? Me[p] : -1;
      if (wloc) {
        if (e < E) wloc[e * C::N3 + p] = (gk >= 0) ? val : 0.0f;
      } else if (gk >= 0) {
        atomicAdd(&w[gk], val);
      }
    }
    __syncthreads();
  }
  cp_async_wait_all();
  if (abort_flag && tid == 0) {  // let the bulk copies still in flight land before the CTA exits
    for (int t = q; t < issued; ++t) wait_group(t);
    atomicExch(err, 1);
  }
}

template <int NP, typename GT>
int launch_ax32_tma(const PmgLevel &lv, const GT *Gp, float h1, float h2, const float *u, float *w, int *err,
                    cudaStream_t st) {
  using C = TmaCfg<NP, GT>;
  if (int rc = ensure_d32(lv.m->device)) return rc;
  auto kern = k_ax32_tma<NP, GT>;
  if (C::SMEM > 48 * 1024) SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
  int per_sm = 0, nsm = 0;
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::THREADS, C::SMEM));
  SEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, lv.m->device));
  const int64_t ngroups = (lv.m->E + C::ELB - 1) / C::ELB;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ngroups, (int64_t)std::max(per_sm, 1) * nsm));
  kern<<<grid, C::THREADS, C::SMEM, st>>>(lv.m->E, lv.Df, Gp, lv.Bf, h1, h2, u, w, lv.map, (float *)lv.m->det_w,
                                           err);
  SEM_LAUNCH_CHECK("k_ax32_tma");
  if (lv.m->det_w) return sem_launch_gather_add_f(lv.m, (const float *)lv.m->det_w, w, st);
  return SEM_OK;
}

template <int NP>
int launch_ax32_np(const PmgLevel &lv, int gprec, float h1, float h2, const float *u, float *w, cudaStream_t st) {
  using C = F32Cfg<NP>;
  if (lv.Gl) {  // N = 7, bfloat16 smoothing: the tensor-core operator
    float *wl = (float *)lv.m->det_w;
    if (int rc = sem_launch_ax_bf16(lv.m, lv.Gl, lv.Ml, lv.Bl, h1, h2, u, w, wl, st)) return rc;
    if (wl) return sem_launch_gather_add_f(lv.m, wl, w, st);
    return SEM_OK;
  }
  if constexpr (NP % 2 == 0 && NP >= 4) {
    if (lv.err) {
      if (gprec == SEM_PREC_BF16) return launch_ax32_tma<NP, __nv_bfloat16>(lv, lv.Gb, h1, h2, u, w, lv.err, st);
      return launch_ax32_tma<NP, float>(lv, lv.Gf, h1, h2, u, w, lv.err, st);
    }
  }
  const unsigned grid = (unsigned)std::max<int64_t>((lv.m->E + C::ELB - 1) / C::ELB, 1);
  float *wloc = (float *)lv.m->det_w;
  if (gprec == SEM_PREC_BF16) {
    auto kern = k_ax32<NP, __nv_bfloat16>;
    if (C::SMEM > 48 * 1024) SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    kern<<<grid, C::THREADS, C::SMEM, st>>>(lv.m->E, lv.Df, lv.Gb, lv.Bf, h1, h2, u, w, lv.map, wloc);
  } else {
    auto kern = k_ax32<NP, float>;
    if (C::SMEM > 48 * 1024) SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    kern<<<grid, C::THREADS, C::SMEM, st>>>(lv.m->E, lv.Df, lv.Gf, lv.Bf, h1, h2, u, w, lv.map, wloc);
  }
  SEM_LAUNCH_CHECK("k_ax32");
  if (wloc) return sem_launch_gather_add_f(lv.m, wloc, w, st);
  return SEM_OK;
}

int launch_ax32(const PmgLevel &lv, int gprec, float h1, float h2, const float *u, float *w, cudaStream_t st) {
  switch (lv.m->n) {
#define CASE(NPV) \
  case NPV:       \
    return launch_ax32_np<NPV>(lv, gprec, h1, h2, u, w, st);
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
#undef CASE
    default:
      return sem_fail(SEM_ERR_INVALID_ARG, "pmg: unsupported order");
  }
}

// ---------------------------------------------------------------- transfers
// One CTA of nf^2 threads per element; thread (i, j) owns the fine column
// (i, j, :). Sum factorisation: nc + nc^2 + nc^3 multiply-adds per column
// stage instead of nc^3 per fine point.
// Fine level uf = P uc (identical values on shared nodes, every copy stores).
// Accumulate form (own != nullptr): uf += P uc and r = b, written by the one
// copy that owns each unique node: the copy whose local index is below N in
// every direction, or N at the last element of a non-periodic direction.
struct Owner {
  int nel[3], per[3];
};
template <typename T>
__global__ void k_prolong(int nf, int nc, int64_t E, const T *__restrict__ J, const int32_t *__restrict__ mapc,
                          const T *__restrict__ uc, const int32_t *__restrict__ mapf, T *__restrict__ uf,
                          int accumulate, Owner ow, const T *__restrict__ bf, T *__restrict__ rf) {
  __shared__ T tile[SEM_MAXNP * SEM_MAXNP * SEM_MAXNP];
  __shared__ T Js[SEM_MAXNP * SEM_MAXNP];
  const int nc3 = nc * nc * nc, nf3 = nf * nf * nf;
  const int tid = threadIdx.x, i = tid % nf, j = tid / nf;
  for (int t = tid; t < nf * nc; t += blockDim.x) Js[t] = J[t];
  for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
    const int64_t ex = e % ow.nel[0], ey = (e / ow.nel[0]) % ow.nel[1], ez = e / ((int64_t)ow.nel[0] * ow.nel[1]);
    __syncthreads();
    for (int t = tid; t < nc3; t += blockDim.x) {
      const int32_t g = mapc[e * nc3 + t];
      tile[t] = g >= 0 ? uc[g] : T(0);
    }
    __syncthreads();
    T t2[SEM_MAXNP];
    for (int c = 0; c < nc; ++c) {
      T sb = T(0);
      for (int b = 0; b < nc; ++b) {
        T sa = T(0);
        for (int a = 0; a < nc; ++a) sa = fma(Js[i * nc + a], tile[a + nc * (b + nc * c)], sa);
        sb = fma(Js[j * nc + b], sa, sb);
      }
      t2[c] = sb;
    }
    for (int k = 0; k < nf; ++k) {
      T s = T(0);
      for (int c = 0; c < nc; ++c) s = fma(Js[k * nc + c], t2[c], s);
      const int32_t g = mapf[e * nf3 + i + nf * (j + nf * k)];
      if (g < 0) continue;
      if (!accumulate) {
        uf[g] = s;
      } else if ((i < nf - 1 || (!ow.per[0] && ex == ow.nel[0] - 1)) &&
                 (j < nf - 1 || (!ow.per[1] && ey == ow.nel[1] - 1)) &&
                 (k < nf - 1 || (!ow.per[2] && ez == ow.nel[2] - 1))) {
        uf[g] += s;
        rf[g] = bf[g];
      }
    }
  }
}

// coarse level rc += R rf = P^T rf: J^T (x) J^T (x) J^T of the fine element's
// rf / multiplicity, summed into the coarse vector
template <typename T>
__global__ void k_restrict(int nf, int nc, int64_t E, const T *__restrict__ J, const int32_t *__restrict__ mapf,
                           const T *__restrict__ minvf, const T *__restrict__ rf,
                           const int32_t *__restrict__ mapc, T *__restrict__ rc, T *__restrict__ wloc) {
  __shared__ T u1[SEM_MAXNP * SEM_MAXNP * SEM_MAXNP];  // [i][j][c]
  __shared__ T u2[SEM_MAXNP * SEM_MAXNP * SEM_MAXNP];  // [i][b][c]
  __shared__ T Js[SEM_MAXNP * SEM_MAXNP];
  const int nc3 = nc * nc * nc, nf3 = nf * nf * nf;
  const int tid = threadIdx.x, i = tid % nf, j = tid / nf;
  for (int t = tid; t < nf * nc; t += blockDim.x) Js[t] = J[t];
  for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
    __syncthreads();
    {
      T v[SEM_MAXNP];
      for (int k = 0; k < nf; ++k) {
        const int32_t g = mapf[e * nf3 + i + nf * (j + nf * k)];
        v[k] = g >= 0 ? rf[g] * minvf[g] : T(0);
      }
      for (int c = 0; c < nc; ++c) {
        T s = T(0);
        for (int k = 0; k < nf; ++k) s = fma(Js[k * nc + c], v[k], s);
        u1[(i * nf + j) * nc + c] = s;
      }
    }
    __syncthreads();
    if (tid < nf * nc) {  // thread (i, b)
      const int ii = tid % nf, b = tid / nf;
      for (int c = 0; c < nc; ++c) {
        T s = T(0);
        for (int jj = 0; jj < nf; ++jj) s = fma(Js[jj * nc + b], u1[(ii * nf + jj) * nc + c], s);
        u2[(ii * nc + b) * nc + c] = s;
      }
    }
    __syncthreads();
    if (tid < nc * nc) {  // thread (a, b)
      const int a = tid % nc, b = tid / nc;
      for (int c = 0; c < nc; ++c) {
        T s = T(0);
        for (int ii = 0; ii < nf; ++ii) s = fma(Js[ii * nc + a], u2[(ii * nc + b) * nc + c], s);
        const int64_t lc = e * nc3 + a + nc * (b + nc * c);
        const int32_t g = mapc[lc];
        if (wloc) wloc[lc] = (g >= 0) ? s : T(0);
        else if (g >= 0) atomicAdd(&rc[g], s);
      }
    }
  }
}

// The same two transfers with the orders fixed at compile time (the (7, 3)
// and (3, 1) level pairs): loops unrolled, J in registers, ELB elements per
// CTA so that a CTA is at least two warps, and the work of the restriction's
// second and third stages spread over all threads. Every output is the same
// sequence of multiply-adds as in k_prolong / k_restrict, so the results are
// bit-identical to theirs.
template <int NF, int NC>
struct XferCfg {
  static constexpr int NT = NF * NF;                    // threads per element
  static constexpr int ELB = NT >= 64 ? 1 : 64 / NT;    // elements per CTA
  static constexpr int THREADS = NT * ELB;
  static constexpr int NC3 = NC * NC * NC, NF3 = NF * NF * NF;
};

template <typename T, int NF, int NC>
__global__ void __launch_bounds__(XferCfg<NF, NC>::THREADS)
    k_prolong_t(int64_t E, const T *__restrict__ Jg, const int32_t *__restrict__ mapc, const T *__restrict__ uc,
                const int32_t *__restrict__ mapf, T *__restrict__ uf, int accumulate, Owner ow,
                const T *__restrict__ bf, T *__restrict__ rf) {
  using C = XferCfg<NF, NC>;
  __shared__ T tile[C::ELB][C::NC3];
  T J[NF][NC];
#pragma unroll
  for (int a = 0; a < NF; ++a)
#pragma unroll
    for (int c = 0; c < NC; ++c) J[a][c] = Jg[a * NC + c];
  const int le = threadIdx.x / C::NT, tid = threadIdx.x - le * C::NT, i = tid % NF, j = tid / NF;
  T Ji[NC], Jj[NC];  // this thread's rows (runtime indices: loaded, not indexed from J)
#pragma unroll
  for (int a = 0; a < NC; ++a) {
    Ji[a] = Jg[i * NC + a];
    Jj[a] = Jg[j * NC + a];
  }
  for (int64_t e0 = (int64_t)blockIdx.x * C::ELB; e0 < E; e0 += (int64_t)gridDim.x * C::ELB) {
    const int64_t e = e0 + le;
    const bool act = e < E;
    int32_t gk[NF];  // the column's fine map entries, loaded before the coarse tile is awaited
#pragma unroll
    for (int k = 0; k < NF; ++k) gk[k] = act ? mapf[e * C::NF3 + i + NF * (j + NF * k)] : -1;
    __syncthreads();
    for (int t = tid; t < C::NC3; t += C::NT) {
      const int32_t g = act ? mapc[e * C::NC3 + t] : -1;
      tile[le][t] = g >= 0 ? uc[g] : T(0);
    }
    __syncthreads();
    if (!act) continue;
    T t2[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T sb = T(0);
#pragma unroll
      for (int b = 0; b < NC; ++b) {
        T sa = T(0);
#pragma unroll
        for (int a = 0; a < NC; ++a) sa = fma(Ji[a], tile[le][a + NC * (b + NC * c)], sa);
        sb = fma(Jj[b], sa, sb);
      }
      t2[c] = sb;
    }
    T sk[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      T s = T(0);
#pragma unroll
      for (int c = 0; c < NC; ++c) s = fma(J[k][c], t2[c], s);
      sk[k] = s;
    }
    if (!accumulate) {
#pragma unroll
      for (int k = 0; k < NF; ++k)
        if (gk[k] >= 0) uf[gk[k]] = sk[k];
      continue;
    }
    const int64_t ex = e % ow.nel[0], ey = (e / ow.nel[0]) % ow.nel[1], ez = e / ((int64_t)ow.nel[0] * ow.nel[1]);
    const bool own_ij = (i < NF - 1 || (!ow.per[0] && ex == ow.nel[0] - 1)) &&
                        (j < NF - 1 || (!ow.per[1] && ey == ow.nel[1] - 1));
    // the owned points' old values and right-hand sides, all loads first
    T uo[NF], bo[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const bool own = gk[k] >= 0 && own_ij && (k < NF - 1 || (!ow.per[2] && ez == ow.nel[2] - 1));
      if (!own) gk[k] = -1;
      uo[k] = own ? uf[gk[k]] : T(0);
      bo[k] = own ? bf[gk[k]] : T(0);
    }
#pragma unroll
    for (int k = 0; k < NF; ++k)
      if (gk[k] >= 0) {
        uf[gk[k]] = uo[k] + sk[k];
        rf[gk[k]] = bo[k];
      }
  }
}

template <typename T, int NF, int NC>
__global__ void __launch_bounds__(XferCfg<NF, NC>::THREADS)
    k_restrict_t(int64_t E, const T *__restrict__ Jg, const int32_t *__restrict__ mapf,
                 const T *__restrict__ minvf, const T *__restrict__ rf, const int32_t *__restrict__ mapc,
                 T *__restrict__ rc, T *__restrict__ wloc) {
  using C = XferCfg<NF, NC>;
  __shared__ T u1[C::ELB][NF * NF * NC];  // [i][j][c]
  __shared__ T u2[C::ELB][NF * NC * NC];  // [i][b][c]
  __shared__ T Js[NF * NC];
  for (int t = threadIdx.x; t < NF * NC; t += C::THREADS) Js[t] = Jg[t];
  T J[NF][NC];
#pragma unroll
  for (int a = 0; a < NF; ++a)
#pragma unroll
    for (int c = 0; c < NC; ++c) J[a][c] = Jg[a * NC + c];
  const int le = threadIdx.x / C::NT, tid = threadIdx.x - le * C::NT, i = tid % NF, j = tid / NF;
  for (int64_t e0 = (int64_t)blockIdx.x * C::ELB; e0 < E; e0 += (int64_t)gridDim.x * C::ELB) {
    const int64_t e = e0 + le;
    const bool act = e < E;
    __syncthreads();
    if (act) {
      T v[NF];
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        const int32_t g = mapf[e * C::NF3 + i + NF * (j + NF * k)];
        v[k] = g >= 0 ? rf[g] * minvf[g] : T(0);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T s = T(0);
#pragma unroll
        for (int k = 0; k < NF; ++k) s = fma(J[k][c], v[k], s);
        u1[le][(i * NF + j) * NC + c] = s;
      }
    }
    __syncthreads();
    if (act) {  // outputs (ii, b, c), spread over the element's threads
#pragma unroll
      for (int o = tid; o < NF * NC * NC; o += C::NT) {
        const int c = o % NC, b = (o / NC) % NC, ii = o / (NC * NC);
        T s = T(0);
#pragma unroll
        for (int jj = 0; jj < NF; ++jj) s = fma(Js[jj * NC + b], u1[le][(ii * NF + jj) * NC + c], s);
        u2[le][(ii * NC + b) * NC + c] = s;
      }
    }
    __syncthreads();
    if (act) {  // outputs (a, b, c)
#pragma unroll
      for (int o = tid; o < C::NC3; o += C::NT) {
        const int a = o % NC, b = (o / NC) % NC, c = o / (NC * NC);
        T s = T(0);
#pragma unroll
        for (int ii = 0; ii < NF; ++ii) s = fma(Js[ii * NC + a], u2[le][(ii * NC + b) * NC + c], s);
        const int64_t lc = e * C::NC3 + a + NC * (b + NC * c);
        const int32_t g = mapc[lc];
        if (wloc) wloc[lc] = (g >= 0) ? s : T(0);
        else if (g >= 0) atomicAdd(&rc[g], s);
      }
    }
  }
}

// Launch the transfer for the level pair (nf, nc): the compile-time kernels
// for the pairs they cover, else the general ones.
template <typename T>
void launch_prolong(int nf, int nc, int64_t E, const T *J, const int32_t *mapc, const T *uc, const int32_t *mapf,
                    T *uf, int accumulate, Owner ow, const T *bf, T *rf, cudaStream_t st) {
  if (nf == 8 && nc == 4) {
    using C = XferCfg<8, 4>;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((E + C::ELB - 1) / C::ELB, 152 * 256));
    k_prolong_t<T, 8, 4><<<grid, C::THREADS, 0, st>>>(E, J, mapc, uc, mapf, uf, accumulate, ow, bf, rf);
  } else if (nf == 4 && nc == 2) {
    using C = XferCfg<4, 2>;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((E + C::ELB - 1) / C::ELB, 152 * 256));
    k_prolong_t<T, 4, 2><<<grid, C::THREADS, 0, st>>>(E, J, mapc, uc, mapf, uf, accumulate, ow, bf, rf);
  } else {
    const unsigned grid = (unsigned)std::min<int64_t>(E, 152 * 256);
    k_prolong<T><<<grid, nf * nf, 0, st>>>(nf, nc, E, J, mapc, uc, mapf, uf, accumulate, ow, bf, rf);
  }
}

template <typename T>
void launch_restrict(int nf, int nc, int64_t E, const T *J, const int32_t *mapf, const T *minvf, const T *rf,
                     const int32_t *mapc, T *rc, T *wloc, cudaStream_t st) {
  if (nf == 8 && nc == 4) {
    using C = XferCfg<8, 4>;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((E + C::ELB - 1) / C::ELB, 152 * 256));
    k_restrict_t<T, 8, 4><<<grid, C::THREADS, 0, st>>>(E, J, mapf, minvf, rf, mapc, rc, wloc);
  } else if (nf == 4 && nc == 2) {
    using C = XferCfg<4, 2>;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((E + C::ELB - 1) / C::ELB, 152 * 256));
    k_restrict_t<T, 4, 2><<<grid, C::THREADS, 0, st>>>(E, J, mapf, minvf, rf, mapc, rc, wloc);
  } else {
    const unsigned grid = (unsigned)std::min<int64_t>(E, 152 * 256);
    k_restrict<T><<<grid, nf * nf, 0, st>>>(nf, nc, E, J, mapf, minvf, rf, mapc, rc, wloc);
  }
}

// ---------------------------------------------------------------- vector kernels
template <typename T>
__global__ void k_cheb_start(int64_t n, const T *__restrict__ b, const T *__restrict__ dinv, T c0,
                             T *__restrict__ x, T *__restrict__ r, T *__restrict__ d) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const T bv = b[g];
    x[g] = T(0);
    r[g] = bv;
    d[g] = c0 * dinv[g] * bv;
  }
}

template <typename T>
__global__ void k_scaled(int64_t n, const T *__restrict__ r, const T *__restrict__ dinv, T c0, T *__restrict__ d) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    d[g] = c0 * dinv[g] * r[g];
}

// x += d;  d = c1 d + c2 dinv r
template <typename T>
__global__ void k_cheb_xd(int64_t n, T c1, T c2, const T *__restrict__ dinv, const T *__restrict__ r, T *__restrict__ x,
                          T *__restrict__ d) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const T dv = d[g];
    x[g] += dv;
    d[g] = c1 * dv + c2 * dinv[g] * r[g];
  }
}

template <typename T>
__global__ void k_axpy_f(int64_t n, T a, const T *__restrict__ x, T *__restrict__ y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    y[g] += a * x[g];
}

template <typename T>
__global__ void k_copy_f(int64_t n, const T *__restrict__ x, T *__restrict__ y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    y[g] = x[g];
}

// binary64 -> binary32 (leading 24 bits) with integer operations only
__global__ void k_d2f(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    b[g] = df::from_f64(a[g]).x;
}

// binary32 -> binary64, exact, with integer operations only
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned fb = __float_as_uint(f);
  const unsigned ef = (fb >> 23) & 0xFFu;
  if (ef == 0u || ef == 255u) return (double)f;  // zero, subnormal, inf, nan: rare
  const unsigned long long hi = (unsigned long long)((fb & 0x80000000u) | ((ef + 896u) << 20) | ((fb & 0x7FFFFFu) >> 3));
  return __longlong_as_double((long long)((hi << 32) | ((unsigned long long)(fb & 7u) << 29)));
}

__global__ void k_f2d(int64_t n, const float *__restrict__ a, double *__restrict__ b) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    b[g] = f2d_bits(a[g]);
}

__global__ void k_g_to_f32(int64_t n, const double *__restrict__ G, float *__restrict__ Gf,
                           __nv_bfloat16 *__restrict__ Gb) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const float v = (float)G[t];  // set-up only
    if (Gf) Gf[t] = v;
    if (Gb) Gb[t] = __float2bfloat16_rn(v);
  }
}

__global__ void k_d2f_plain(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    b[g] = (float)a[g];  // set-up only
}

template <typename T>
__global__ void k_minv(int64_t n, const double *__restrict__ mult, T *__restrict__ minv) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    minv[g] = (T)(1.0 / mult[g]);
}

// alternating lattice vector (-1)^(I+J+K) on free nodes
template <typename T>
__global__ void k_alt(int64_t n, int64_t nx, int64_t ny, const uint8_t *__restrict__ mask, T *__restrict__ v) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = g % nx, J = (g / nx) % ny, K = g / (nx * ny);
    v[g] = (!mask || mask[g]) ? (((I + J + K) & 1) ? T(-1) : T(1)) : T(0);
  }
}

// Degree-2 Chebyshev smoothing with fused vector passes (c1 = 1/5,
// c2 = 12/(5 lam) of the recurrence); the same roundings as the general path.
// pre, part 1: b (from binary64 when b64 is given), r = b, d = c0 dinv b
__global__ void k_pre2a(int64_t n, const double *__restrict__ b64, float *__restrict__ b, const float *__restrict__ dinv,
                        float c0, float *__restrict__ r, float *__restrict__ d) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    float bv;
    if (b64) {
      bv = df::from_f64(b64[g]).x;
      b[g] = bv;
    } else {
      bv = b[g];
    }
    r[g] = bv;
    d[g] = c0 * dinv[g] * bv;
  }
}

// pre, part 2 (r = b - A d): x = d + (c1 d + c2 dinv r), then r = b for the residual
__global__ void k_pre2b(int64_t n, float c1, float c2, const float *__restrict__ dinv, const float *__restrict__ b,
                        float *__restrict__ r, const float *__restrict__ d, float *__restrict__ x) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const float dv = d[g];
    const float d1 = c1 * dv + c2 * dinv[g] * r[g];
    x[g] = 0.0f + dv + d1;
    r[g] = b[g];
  }
}

// post (r = b - A x - A d): x = (x + d) + (c1 d + c2 dinv r); written to z64 in binary64 when given
__global__ void k_post2(int64_t n, float c1, float c2, const float *__restrict__ dinv, const float *__restrict__ r,
                        const float *__restrict__ d, float *__restrict__ x, double *__restrict__ z64) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const float dv = d[g];
    const float d1 = c1 * dv + c2 * dinv[g] * r[g];
    const float xv = (x[g] + dv) + d1;
    if (z64) z64[g] = f2d_bits(xv);
    else x[g] = xv;
  }
}

// y = a x
template <typename T>
__global__ void k_copy_scale_f(int64_t n, T a, const T *__restrict__ x, T *__restrict__ y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    y[g] = a * x[g];
}

// w = dinv * w (in place), partial sums of w.w and v.v (binary32 per thread,
// binary64 across threads: an eigenvalue estimate needs no more)
template <typename T>
__global__ void k_power_step(int64_t n, const T *__restrict__ dinv, T *__restrict__ w, const T *__restrict__ v,
                             double *__restrict__ part) {
  __shared__ double red[2][32];
  T wwf = T(0), vvf = T(0);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const T x = dinv[g] * w[g];
    w[g] = x;
    wwf = fma(x, x, wwf);
    vvf = fma(v[g], v[g], vvf);
  }
  double ww = wwf, vv = vvf;
  for (int off = 16; off > 0; off >>= 1) {
    ww += __shfl_xor_sync(0xffffffffu, ww, off);
    vv += __shfl_xor_sync(0xffffffffu, vv, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ww;
    red[1][threadIdx.x >> 5] = vv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) {
      a += red[0][t];
      b += red[1][t];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}


// partial sums of (a.b, c.d) in binary64; c may be null
__global__ void k_dots(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                       const double *__restrict__ c, const double *__restrict__ d, double *__restrict__ part) {
  __shared__ double red[2][32];
  double s0 = 0.0, s1 = 0.0;
  // four nodes per pass with their loads issued first (kPart CTAs leave too
  // few loads in flight otherwise); each thread keeps the plain loop's order
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; g + 3 * S < n; g += 4 * S) {
    double av[4], bv[4], cv[4], dv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      av[u] = a[g + u * S];
      bv[u] = b[g + u * S];
      if (c) {
        cv[u] = c[g + u * S];
        dv[u] = d[g + u * S];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      s0 = fma(av[u], bv[u], s0);
      if (c) s1 = fma(cv[u], dv[u], s1);
    }
  }
  for (; g < n; g += S) {
    s0 = fma(a[g], b[g], s0);
    if (c) s1 = fma(c[g], d[g], s1);
  }
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s0;
    red[1][threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0, y = 0;
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) {
      x += red[0][t];
      y += red[1][t];
    }
    part[2 * blockIdx.x] = x;
    part[2 * blockIdx.x + 1] = y;
  }
}

// x += alpha p; r -= alpha w; and the partial sums of r.r of the new r.
// Launched on kPart blocks of 256 threads, it visits the nodes in the order of
// k_dots and sums the same way, so the partials are the bits k_dots(r, r)
// would give (one pass over r less per iteration).
__global__ void k_fcg_update(int64_t n, double alpha, const double *__restrict__ p, const double *__restrict__ w,
                             double *__restrict__ x, double *__restrict__ r, double *__restrict__ part) {
  __shared__ double red[32];
  double s0 = 0.0;
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; g + 3 * S < n; g += 4 * S) {  // four nodes per pass, loads first (as in k_dots)
    double pv[4], wv[4], xv[4], rv0[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      pv[u] = p[g + u * S];
      wv[u] = w[g + u * S];
      xv[u] = x[g + u * S];
      rv0[u] = r[g + u * S];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x[g + u * S] = fma(alpha, pv[u], xv[u]);
      const double rv = fma(-alpha, wv[u], rv0[u]);
      r[g + u * S] = rv;
      s0 = fma(rv, rv, s0);
    }
  }
  for (; g < n; g += S) {
    x[g] = fma(alpha, p[g], x[g]);
    const double rv = fma(-alpha, w[g], r[g]);
    r[g] = rv;
    s0 = fma(rv, rv, s0);
  }
  for (int off = 16; off > 0; off >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0;
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) v += red[t];
    part[2 * blockIdx.x] = v;
    part[2 * blockIdx.x + 1] = 0.0;
  }
}

// p = z + beta p; w = 0 for the next operator application (no separate
// clearing pass)
__global__ void k_xpby(int64_t n, const double *__restrict__ z, double beta, double *__restrict__ p,
                       double *__restrict__ w) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    p[g] = fma(beta, p[g], z[g]);
    w[g] = 0.0;
  }
}

// r = M b; x = 0 unless the solve starts from the guess held in x
__global__ void k_init_fcg(int64_t n, const double *__restrict__ b, const uint8_t *__restrict__ mask,
                           double *__restrict__ x, double *__restrict__ r, int keep_x) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    if (!keep_x) x[g] = 0.0;
    r[g] = (!mask || mask[g]) ? b[g] : 0.0;
  }
}

__global__ void k_sub_from(int64_t n, const double *__restrict__ w, double *__restrict__ r) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    r[g] -= w[g];
}

// ---------------------------------------------------------------- host helpers
// fixed-order sum of n partials into *out (one CTA of 1024 threads); for the
// outer operator's many p.w partials, first summed in chunks by k_sum_chunks
constexpr int kSumThreads = 1024;
__global__ void __launch_bounds__(256) k_sum_chunks(const double *__restrict__ part, int n, int chunk,
                                                    double *__restrict__ out) {
  __shared__ double red[8];
  const int b0 = blockIdx.x * chunk, m = min(chunk, n - b0);
  double v = 0.0;
  for (int t = threadIdx.x; t < m; t += 256) v += part[b0 + t];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    out[blockIdx.x] = s;
  }
}
__global__ void __launch_bounds__(kSumThreads) k_sum_fixed(const double *__restrict__ part, int n,
                                                           double *__restrict__ out) {
  __shared__ double red[kSumThreads / 32];
  double v = 0.0;
  for (int t = threadIdx.x; t < n; t += kSumThreads) v += part[t];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kSumThreads / 32; ++w) s += red[w];
    *out = s;
  }
}

int sum_pairs(const double *dpart, double *a, double *b, cudaStream_t st) {
  double h[2 * kPart];
  SEM_CUDA(cudaMemcpyAsync(h, dpart, sizeof(h), cudaMemcpyDeviceToHost, st));
  SEM_CUDA(cudaStreamSynchronize(st));
  double x = 0, y = 0;
  for (int t = 0; t < kPart; ++t) {
    x += h[2 * t];
    y += h[2 * t + 1];
  }
  *a = x;
  *b = y;
  return SEM_OK;
}

template <typename T>
int interp_matrix(const sem_mesh *mf, const sem_mesh *mc, T *dJ, cudaStream_t st) {
  const int nf = mf->n, nc = mc->n;
  std::vector<T> J(nf * nc);
  for (int i = 0; i < nf; ++i)
    for (int m = 0; m < nc; ++m) {
      long double v = 1.0L;
      for (int j = 0; j < nc; ++j)
        if (j != m) v *= ((long double)mf->xi[i] - mc->xi[j]) / ((long double)mc->xi[m] - mc->xi[j]);
      J[i * nc + m] = (T)v;
    }
  SEM_CUDA(cudaMemcpyAsync(dJ, J.data(), sizeof(T) * nf * nc, cudaMemcpyHostToDevice, st));
  SEM_CUDA(cudaStreamSynchronize(st));  // J lives on the host stack frame until copied
  return SEM_OK;
}

int ax32(sem_pmg *P, int l, float h1s, const float *u, float *w, cudaStream_t st) {
  return launch_ax32(P->L[l], P->o.smoother_precision, (float)(h1s * P->h1), (float)(h1s * P->h2), u, w, st);
}

// r = b - A x
int residual(sem_pmg *P, int l, cudaStream_t st) {
  PmgLevel &lv = P->L[l];
  const int64_t n = lv.m->n_unique;
  k_copy_f<float><<<grid_for(n, 256), 256, 0, st>>>(n, lv.b, lv.r);
  return ax32(P, l, -1.0f, lv.x, lv.r, st);
}

// Chebyshev smoothing of A x = b on level l; zero initial guess when `zero`
int smooth(sem_pmg *P, int l, bool zero, cudaStream_t st) {
  PmgLevel &lv = P->L[l];
  const int64_t n = lv.m->n_unique;
  const unsigned g = grid_for(n, 256);
  const float lam = lv.lam;
  const float c0 = 4.0f / (3.0f * lam);
  int rc;
  if (zero) {
    k_cheb_start<float><<<g, 256, 0, st>>>(n, lv.b, lv.dinv, c0, lv.x, lv.r, lv.d);
  } else {
    if ((rc = residual(P, l, st))) return rc;
    k_scaled<float><<<g, 256, 0, st>>>(n, lv.r, lv.dinv, c0, lv.d);
  }
  for (int i = 1; i < P->o.cheb_degree; ++i) {
    if ((rc = ax32(P, l, -1.0f, lv.d, lv.r, st))) return rc;  // r -= A d
    const float c1 = (float)(2 * i - 1) / (float)(2 * i + 3);
    const float c2 = (float)(8 * i + 4) / ((float)(2 * i + 3) * lam);
    k_cheb_xd<float><<<g, 256, 0, st>>>(n, c1, c2, lv.dinv, lv.r, lv.x, lv.d);
  }
  k_axpy_f<float><<<g, 256, 0, st>>>(n, 1.0f, lv.d, lv.x);
  SEM_LAUNCH_CHECK("chebyshev");
  return SEM_OK;
}

int restrict_to(sem_pmg *P, int l, const float *rf, float *rc, cudaStream_t st) {
  PmgLevel &f = P->L[l], &c = P->L[l + 1];
  SEM_CUDA(cudaMemsetAsync(rc, 0, sizeof(float) * c.m->n_unique, st));
  float *wloc = (float *)c.m->det_w;
  launch_restrict<float>(f.m->n, c.m->n, f.m->E, P->J[l], f.map, f.minv, rf, c.map, rc, wloc, st);
  SEM_LAUNCH_CHECK("k_restrict");
  if (wloc) return sem_launch_gather_add_f(c.m, wloc, rc, st);
  return SEM_OK;
}

Owner owner_of(const sem_mesh *m) {
  Owner o;
  for (int d = 0; d < 3; ++d) {
    o.nel[d] = m->nel[d];
    o.per[d] = m->periodic[d];
  }
  return o;
}

int prolong_to(sem_pmg *P, int l, const float *uc, float *uf, cudaStream_t st) {
  PmgLevel &f = P->L[l], &c = P->L[l + 1];
  SEM_CUDA(cudaMemsetAsync(uf, 0, sizeof(float) * f.m->n_unique, st));
  launch_prolong<float>(f.m->n, c.m->n, f.m->E, P->J[l], c.map, uc, f.map, uf, 0, owner_of(f.m), nullptr, nullptr, st);
  SEM_LAUNCH_CHECK("k_prolong");
  return SEM_OK;
}

// x += P uc and r = b on level l (each unique node once, by its owner copy)
int prolong_add(sem_pmg *P, int l, const float *uc, float *x, const float *b, float *r, cudaStream_t st) {
  PmgLevel &f = P->L[l], &c = P->L[l + 1];
  launch_prolong<float>(f.m->n, c.m->n, f.m->E, P->J[l], c.map, uc, f.map, x, 1, owner_of(f.m), b, r, st);
  SEM_LAUNCH_CHECK("k_prolong (accumulate)");
  return SEM_OK;
}

// subtract the mean of a binary64 vector (fixed-order partials, device scalar)
__global__ void k_mean_part(int64_t n, const double *__restrict__ x, double *__restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    s += x[g];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_sub_mean(int64_t n, int np, const double *__restrict__ part, double *__restrict__ x) {
  __shared__ double mean;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < np; ++b) t += part[b];
    mean = t / (double)n;
  }
  __syncthreads();
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    x[g] -= mean;
}

int remove_mean_d(sem_pmg *P, double *x, int64_t n, cudaStream_t st) {
  k_mean_part<<<kPart, 256, 0, st>>>(n, x, P->part);
  k_sub_mean<<<grid_for(n, 256), 256, 0, st>>>(n, kPart, P->part, x);
  SEM_LAUNCH_CHECK("remove mean");
  return SEM_OK;
}

int coarse_solve(sem_pmg *P, cudaStream_t st) {
  PmgLevel &lv = P->L.back();
  const int64_t n = lv.m->n_unique;
  k_f2d<<<grid_for(n, 256), 256, 0, st>>>(n, lv.b, P->cb);
  if (P->o.mask_mode) {  // singular Neumann problem: make the right-hand side consistent
    if (int rc = remove_mean_d(P, P->cb, n, st)) return rc;
  }
  int rc;
  if (P->cdinv) {  // N = 1 element matrices, atomic assembly: one persistent launch
    rc = sem_pcg_n1_persistent(lv.m, P->h1, P->h2, P->cb, P->cx, P->cdinv, lv.map, P->o.coarse_tol,
                               P->o.coarse_maxit, P->cws, nullptr, nullptr, st);
  } else {
    sem_solver_opts o;
  o.initial_guess = 0;
    o.tol = P->o.coarse_tol;
    o.maxit = P->o.coarse_maxit;
    o.precision = SEM_PREC_DF64;  // binary64-accurate; native FP64 is pipe-bound even at N = 1
    o.timeout_s = 0.0;
    o.mask_mode = P->o.mask_mode;
    sem_solve_stats stt;
    rc = sem_pcg_solve_ex(lv.m, P->h1, P->h2, P->cb, P->cx, &o, P->cws, &stt, (void *)st, 8);
  }
  if (rc && rc != SEM_ERR_NOT_CONVERGED) return rc;
  k_d2f<<<grid_for(n, 256), 256, 0, st>>>(n, P->cx, lv.x);
  SEM_LAUNCH_CHECK("coarse solve");
  return SEM_OK;
}

// V-cycle on level l: L[l].x ~ A_l^{-1} L[l].b
int vcycle(sem_pmg *P, int l, cudaStream_t st) {
  if (l == (int)P->L.size() - 1) return coarse_solve(P, st);
  int rc;
  PmgLevel &lv = P->L[l];
  const int64_t n = lv.m->n_unique;
  if ((rc = smooth(P, l, true, st))) return rc;
  if ((rc = residual(P, l, st))) return rc;
  if ((rc = restrict_to(P, l, lv.r, P->L[l + 1].b, st))) return rc;
  if ((rc = vcycle(P, l + 1, st))) return rc;
  if ((rc = prolong_to(P, l, P->L[l + 1].x, lv.t, st))) return rc;
  k_axpy_f<float><<<grid_for(n, 256), 256, 0, st>>>(n, 1.0f, lv.t, lv.x);
  return smooth(P, l, false, st);
}

// The V-cycle for degree-2 smoothing with fused vector passes (the same
// operations in the same order as vcycle; 8 instead of 17 streaming passes
// over the level's vectors). Level 0 may read its right-hand side in binary64
// (in64) and write the correction in binary64 (out64).
int vcycle2(sem_pmg *P, int l, cudaStream_t st, const double *in64, double *out64) {
  if (l == (int)P->L.size() - 1) return coarse_solve(P, st);
  int rc;
  PmgLevel &lv = P->L[l];
  const int64_t n = lv.m->n_unique;
  const unsigned g = grid_for(n, 256);
  const float lam = lv.lam;
  const float c0 = 4.0f / (3.0f * lam);
  const float c1 = 1.0f / 5.0f, c2 = 12.0f / (5.0f * lam);
  k_pre2a<<<g, 256, 0, st>>>(n, in64, lv.b, lv.dinv, c0, lv.r, lv.d);
  if ((rc = ax32(P, l, -1.0f, lv.d, lv.r, st))) return rc;  // r = b - A d
  k_pre2b<<<g, 256, 0, st>>>(n, c1, c2, lv.dinv, lv.b, lv.r, lv.d, lv.x);
  SEM_LAUNCH_CHECK("pre-smoothing");
  if ((rc = ax32(P, l, -1.0f, lv.x, lv.r, st))) return rc;  // r = b - A x
  if ((rc = restrict_to(P, l, lv.r, P->L[l + 1].b, st))) return rc;
  if ((rc = vcycle2(P, l + 1, st, nullptr, nullptr))) return rc;
  if ((rc = prolong_add(P, l, P->L[l + 1].x, lv.x, lv.b, lv.r, st))) return rc;  // x += P xc, r = b
  if ((rc = ax32(P, l, -1.0f, lv.x, lv.r, st))) return rc;                       // r = b - A x
  k_scaled<float><<<g, 256, 0, st>>>(n, lv.r, lv.dinv, c0, lv.d);
  if ((rc = ax32(P, l, -1.0f, lv.d, lv.r, st))) return rc;  // r -= A d
  k_post2<<<g, 256, 0, st>>>(n, c1, c2, lv.dinv, lv.r, lv.d, lv.x, out64);
  SEM_LAUNCH_CHECK("post-smoothing");
  return SEM_OK;
}

// ---------------------------------------------------------------- binary64-accurate smoothing
// The same V-cycle with every smoothing level in binary64 vectors and the
// double-float operator (SEM_PREC_DF64): the reference against which the
// binary32 / bfloat16 smoothing shows what the lower precision costs.
// w += h1s (h1 A + h2 B) u on level l
int ax64(sem_pmg *P, int l, double h1s, const double *u, double *w, cudaStream_t st) {
  PmgLevel &lv = P->L[l];
  return sem_launch_ax_assembled(lv.m, h1s * P->h1, h1s * P->h2, u, w, nullptr, SEM_PREC_DF64, st, lv.map);
}

int residual64(sem_pmg *P, int l, cudaStream_t st) {
  PmgLevel &lv = P->L[l];
  const int64_t n = lv.m->n_unique;
  k_copy_f<double><<<grid_for(n, 256), 256, 0, st>>>(n, lv.b64, lv.r64);
  return ax64(P, l, -1.0, lv.x64, lv.r64, st);
}

int smooth64(sem_pmg *P, int l, bool zero, cudaStream_t st) {
  PmgLevel &lv = P->L[l];
  const int64_t n = lv.m->n_unique;
  const unsigned g = grid_for(n, 256);
  const double lam = lv.lam64;
  const double c0 = 4.0 / (3.0 * lam);
  int rc;
  if (zero) {
    k_cheb_start<double><<<g, 256, 0, st>>>(n, lv.b64, lv.dinv64, c0, lv.x64, lv.r64, lv.d64);
  } else {
    if ((rc = residual64(P, l, st))) return rc;
    k_scaled<double><<<g, 256, 0, st>>>(n, lv.r64, lv.dinv64, c0, lv.d64);
  }
  for (int i = 1; i < P->o.cheb_degree; ++i) {
    if ((rc = ax64(P, l, -1.0, lv.d64, lv.r64, st))) return rc;  // r -= A d
    const double c1 = (double)(2 * i - 1) / (double)(2 * i + 3);
    const double c2 = (double)(8 * i + 4) / ((double)(2 * i + 3) * lam);
    k_cheb_xd<double><<<g, 256, 0, st>>>(n, c1, c2, lv.dinv64, lv.r64, lv.x64, lv.d64);
  }
  k_axpy_f<double><<<g, 256, 0, st>>>(n, 1.0, lv.d64, lv.x64);
  SEM_LAUNCH_CHECK("chebyshev (binary64)");
  return SEM_OK;
}

int restrict64(sem_pmg *P, int l, const double *rf, double *rc, cudaStream_t st) {
  PmgLevel &f = P->L[l], &c = P->L[l + 1];
  SEM_CUDA(cudaMemsetAsync(rc, 0, sizeof(double) * c.m->n_unique, st));
  double *wloc = (double *)c.m->det_w;
  launch_restrict<double>(f.m->n, c.m->n, f.m->E, P->J64[l], f.map, f.minv64, rf, c.map, rc, wloc, st);
  SEM_LAUNCH_CHECK("k_restrict (binary64)");
  if (wloc) return sem_launch_gather_add(c.m, wloc, rc, st);
  return SEM_OK;
}

int prolong64(sem_pmg *P, int l, const double *uc, double *uf, cudaStream_t st) {
  PmgLevel &f = P->L[l], &c = P->L[l + 1];
  SEM_CUDA(cudaMemsetAsync(uf, 0, sizeof(double) * f.m->n_unique, st));
  launch_prolong<double>(f.m->n, c.m->n, f.m->E, P->J64[l], c.map, uc, f.map, uf, 0, owner_of(f.m), nullptr, nullptr,
                         st);
  SEM_LAUNCH_CHECK("k_prolong (binary64)");
  return SEM_OK;
}

// the coarsest level reads P->cb and writes P->cx directly (its b64 / x64)
int coarse_solve64(sem_pmg *P, cudaStream_t st) {
  PmgLevel &lv = P->L.back();
  const int64_t n = lv.m->n_unique;
  if (P->o.mask_mode)
    if (int rc = remove_mean_d(P, P->cb, n, st)) return rc;
  int rc;
  if (P->cdinv) {
    rc = sem_pcg_n1_persistent(lv.m, P->h1, P->h2, P->cb, P->cx, P->cdinv, lv.map, P->o.coarse_tol,
                               P->o.coarse_maxit, P->cws, nullptr, nullptr, st);
  } else {
    sem_solver_opts o;
  o.initial_guess = 0;
    o.tol = P->o.coarse_tol;
    o.maxit = P->o.coarse_maxit;
    o.precision = SEM_PREC_DF64;
    o.timeout_s = 0.0;
    o.mask_mode = P->o.mask_mode;
    sem_solve_stats stt;
    rc = sem_pcg_solve_ex(lv.m, P->h1, P->h2, P->cb, P->cx, &o, P->cws, &stt, (void *)st, 8);
  }
  return (rc && rc != SEM_ERR_NOT_CONVERGED) ? rc : SEM_OK;
}

int vcycle64(sem_pmg *P, int l, cudaStream_t st) {
  if (l == (int)P->L.size() - 1) return coarse_solve64(P, st);
  int rc;
  PmgLevel &lv = P->L[l];
  const int64_t n = lv.m->n_unique;
  if ((rc = smooth64(P, l, true, st))) return rc;
  if ((rc = residual64(P, l, st))) return rc;
  if ((rc = restrict64(P, l, lv.r64, P->L[l + 1].b64, st))) return rc;
  if ((rc = vcycle64(P, l + 1, st))) return rc;
  if ((rc = prolong64(P, l, P->L[l + 1].x64, lv.t64, st))) return rc;
  k_axpy_f<double><<<grid_for(n, 256), 256, 0, st>>>(n, 1.0, lv.t64, lv.x64);
  return smooth64(P, l, false, st);
}

int power_lambda64(sem_pmg *P, int l, cudaStream_t st) {
  PmgLevel &lv = P->L[l];
  const sem_mesh *m = lv.m;
  const int64_t n = m->n_unique;
  const int64_t nx = (int64_t)m->nel[0] * m->N + (m->periodic[0] ? 0 : 1);
  const int64_t ny = (int64_t)m->nel[1] * m->N + (m->periodic[1] ? 0 : 1);
  k_alt<double><<<grid_for(n, 256), 256, 0, st>>>(n, nx, ny, P->o.mask_mode ? nullptr : m->mask, lv.x64);
  double lam = 0.0;
  for (int it = 0; it < P->o.power_its; ++it) {
    SEM_CUDA(cudaMemsetAsync(lv.t64, 0, sizeof(double) * n, st));
    if (int rc = ax64(P, l, 1.0, lv.x64, lv.t64, st)) return rc;
    k_power_step<double><<<kPart, 256, 0, st>>>(n, lv.dinv64, lv.t64, lv.x64, P->part);
    SEM_LAUNCH_CHECK("power iteration (binary64)");
    double ww, vv;
    if (int rc = sum_pairs(P->part, &ww, &vv, st)) return rc;
    if (!(ww > 0.0) || !(vv > 0.0)) return sem_fail(SEM_ERR_BREAKDOWN, "pmg: power iteration degenerated");
    lam = sqrt(ww / vv);
    k_copy_scale_f<double><<<grid_for(n, 256), 256, 0, st>>>(n, 1.0 / sqrt(ww), lv.t64, lv.x64);
  }
  lv.lam64 = P->o.lambda_safety * lam;
  lv.lam = (float)lv.lam64;
  return SEM_OK;
}

int power_lambda(sem_pmg *P, int l, cudaStream_t st) {
  PmgLevel &lv = P->L[l];
  const sem_mesh *m = lv.m;
  const int64_t n = m->n_unique;
  const int64_t nx = (int64_t)m->nel[0] * m->N + (m->periodic[0] ? 0 : 1);
  const int64_t ny = (int64_t)m->nel[1] * m->N + (m->periodic[1] ? 0 : 1);
  k_alt<float><<<grid_for(n, 256), 256, 0, st>>>(n, nx, ny, P->o.mask_mode ? nullptr : m->mask, lv.x);
  double lam = 0.0;
  for (int it = 0; it < P->o.power_its; ++it) {
    SEM_CUDA(cudaMemsetAsync(lv.t, 0, sizeof(float) * n, st));
    if (int rc = ax32(P, l, 1.0f, lv.x, lv.t, st)) return rc;
    k_power_step<float><<<kPart, 256, 0, st>>>(n, lv.dinv, lv.t, lv.x, P->part);
    SEM_LAUNCH_CHECK("power iteration");
    double ww, vv;
    if (int rc = sum_pairs(P->part, &ww, &vv, st)) return rc;
    if (!(ww > 0.0) || !(vv > 0.0)) return sem_fail(SEM_ERR_BREAKDOWN, "pmg: power iteration degenerated");
    lam = sqrt(ww / vv);
    k_copy_scale_f<float><<<grid_for(n, 256), 256, 0, st>>>(n, (float)(1.0 / sqrt(ww)), lv.t, lv.x);
  }
  lv.lam = (float)(P->o.lambda_safety * lam);
  return SEM_OK;
}

void free_pmg(sem_pmg *P) {
  if (!P) return;
  for (auto &lv : P->L)
    if (lv.own && lv.m) sem_mesh_destroy(lv.m);
  for (void *q : P->owned) cudaFree(q);
  delete P;
}

}  // namespace

namespace {
// read and clear the persistent operator's error flag (synchronises the stream)
int check_err(sem_pmg *P, cudaStream_t st) {
  int h = 0;
  SEM_CUDA(cudaMemcpyAsync(&h, P->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SEM_CUDA(cudaStreamSynchronize(st));
  if (h) {
    cudaMemsetAsync(P->err, 0, sizeof(int), st);
    return sem_fail(SEM_ERR_CUDA, "pmg: a bulk shared-memory copy did not complete within its wait limit");
  }
  return SEM_OK;
}
}  // namespace

extern "C" int sem_pmg_create(const sem_mesh *m, double h1, double h2, const sem_pmg_opts *o, void *stream,
                              sem_pmg **out) {
  if (!m || !o || !out) return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_create: NULL argument");
  *out = nullptr;
  if (m->slab) return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_create: needs the whole box, not a partition's slab mesh");
  if (o->nlevels < 2 || o->nlevels > 4 || o->orders[0] != m->N)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_create: need 2..4 levels with orders[0] = the mesh's N");
  for (int l = 1; l < o->nlevels; ++l)
    if (o->orders[l] < 1 || o->orders[l] >= o->orders[l - 1])
      return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_create: orders must decrease strictly and stay >= 1");
  if (o->smoother_precision != SEM_PREC_FP32 && o->smoother_precision != SEM_PREC_BF16 &&
      o->smoother_precision != SEM_PREC_DF64)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_create: smoother precision must be FP32, BF16 or DF64");
  const bool p64 = o->smoother_precision == SEM_PREC_DF64;
  if (o->mask_mode != 0 && o->mask_mode != 1) return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_create: bad mask_mode");
  if (o->cheb_degree < 1 || !(o->lambda_safety >= 1.0) || o->power_its < 1 || !(o->coarse_tol > 0) ||
      o->coarse_maxit < 1 || !(h1 > 0) || !(h2 >= 0))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_create: bad option value");
  cudaStream_t st = as_stream(stream);
  sem_pmg *P = new sem_pmg();
  P->o = *o;
  P->h1 = h1;
  P->h2 = h2;
  int rc = SEM_OK;
  auto alloc = [&](void **p, size_t bytes) -> int {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return sem_cuda_fail(e, "sem_pmg_create: cudaMalloc");
    P->owned.push_back(*p);
    return SEM_OK;
  };
  P->L.resize(o->nlevels);
  for (int l = 0; l < o->nlevels && !rc; ++l) {
    PmgLevel &lv = P->L[l];
    if (l == 0) {
      lv.m = const_cast<sem_mesh *>(m);
    } else {
      sem_box_desc d = m->desc;
      d.N = o->orders[l];
      if (o->mask_mode)
        for (int f = 0; f < 6; ++f) d.dirichlet[f] = 0;
      rc = sem_mesh_create_box(&d, stream, &lv.m);
      if (rc) break;
      lv.own = true;
      if (m->det_w && (rc = sem_mesh_set_deterministic(lv.m, 1))) break;
    }
    lv.map = o->mask_mode ? lv.m->l2g : lv.m->l2gm;
    const int64_t nL = lv.m->n_local, nU = lv.m->n_unique;
    const bool coarsest = l == o->nlevels - 1;
    if (p64) {  // binary64 level vectors; the coarsest level's are the coarse solve's (set below)
      if (!coarsest) {
        double **v64[] = {&lv.b64, &lv.x64, &lv.r64, &lv.d64, &lv.t64, &lv.dinv64, &lv.minv64};
        for (double **v : v64) rc = rc ? rc : alloc((void **)v, sizeof(double) * nU);
      }
      continue;
    }
    if (!coarsest) {
      if (o->smoother_precision == SEM_PREC_BF16 && lv.m->n == 8) {  // N = 7: bfloat16 tensor-core operator
        rc = rc ? rc : alloc(&lv.Gl, sem_bf16_layout_bytes(lv.m, 0));
        rc = rc ? rc : alloc(&lv.Ml, sem_bf16_layout_bytes(lv.m, 1));
        if (h2 != 0.0) rc = rc ? rc : alloc(&lv.Bl, sem_bf16_layout_bytes(lv.m, 1));
      } else if (o->smoother_precision == SEM_PREC_BF16) {
        rc = rc ? rc : alloc((void **)&lv.Gb, sizeof(__nv_bfloat16) * 6 * nL);
      } else {
        rc = rc ? rc : alloc((void **)&lv.Gf, sizeof(float) * 6 * nL);
      }
      rc = rc ? rc : alloc((void **)&lv.Bf, sizeof(float) * nL);
      rc = rc ? rc : alloc((void **)&lv.Df, sizeof(float) * lv.m->n * lv.m->n);
      rc = rc ? rc : alloc((void **)&lv.dinv, sizeof(float) * nU);
      rc = rc ? rc : alloc((void **)&lv.r, sizeof(float) * nU);
      rc = rc ? rc : alloc((void **)&lv.d, sizeof(float) * nU);
      rc = rc ? rc : alloc((void **)&lv.t, sizeof(float) * nU);
      rc = rc ? rc : alloc((void **)&lv.minv, sizeof(float) * nU);
    }
    rc = rc ? rc : alloc((void **)&lv.b, sizeof(float) * nU);
    rc = rc ? rc : alloc((void **)&lv.x, sizeof(float) * nU);
  }
  if (!rc) rc = alloc((void **)&P->part, sizeof(double) * 2 * kPart);
  if (!rc) rc = alloc((void **)&P->err, sizeof(int));
  if (rc) {
    free_pmg(P);
    return rc;
  }
  cudaMemsetAsync(P->err, 0, sizeof(int), st);
  for (int l = 0; l + 1 < o->nlevels; ++l) P->L[l].err = P->err;
  // per-level binary64 data (binary64-accurate smoothing)
  for (int l = 0; p64 && l + 1 < o->nlevels && !rc; ++l) {
    PmgLevel &lv = P->L[l];
    const sem_mesh *lm = lv.m;
    k_minv<double><<<grid_for(lm->n_unique, 256), 256, 0, st>>>(lm->n_unique, lm->mult, lv.minv64);
    rc = sem_jacobi_inv_mode(lm, h1, h2, o->mask_mode ? 0 : 1, lv.dinv64, st);
    if (!rc) rc = power_lambda64(P, l, st);
  }
  // per-level binary32 data
  for (int l = 0; !p64 && l + 1 < o->nlevels && !rc; ++l) {
    PmgLevel &lv = P->L[l];
    const sem_mesh *lm = lv.m;
    if (lv.Gl) rc = sem_bf16_pack(lm, lv.map, lv.Gl, lv.Ml, lv.Bl, st);
    else k_g_to_f32<<<grid_for(6 * lm->n_local, 256), 256, 0, st>>>(6 * lm->n_local, lm->G, lv.Gf, lv.Gb);
    if (rc) break;
    k_d2f_plain<<<grid_for(lm->n_local, 256), 256, 0, st>>>(lm->n_local, lm->B, lv.Bf);
    k_d2f_plain<<<1, 128, 0, st>>>(lm->n * lm->n, lm->dD, lv.Df);
    k_minv<float><<<grid_for(lm->n_unique, 256), 256, 0, st>>>(lm->n_unique, lm->mult, lv.minv);
    // Jacobi diagonal (binary64) -> binary32
    double *dd = nullptr;
    if (cudaMalloc(&dd, sizeof(double) * lm->n_unique) != cudaSuccess) {
      rc = sem_fail(SEM_ERR_NOMEM, "sem_pmg_create: cudaMalloc(diag)");
      break;
    }
    rc = sem_jacobi_inv_mode(lm, h1, h2, o->mask_mode ? 0 : 1, dd, st);
    k_d2f_plain<<<grid_for(lm->n_unique, 256), 256, 0, st>>>(lm->n_unique, dd, lv.dinv);
    cudaStreamSynchronize(st);
    cudaFree(dd);
    if (!rc) rc = power_lambda(P, l, st);
  }
  for (int l = 0; l + 1 < o->nlevels && !rc; ++l) {
    rc = alloc((void **)&P->J[l], sizeof(float) * P->L[l].m->n * P->L[l + 1].m->n);
    if (!rc) rc = interp_matrix<float>(P->L[l].m, P->L[l + 1].m, P->J[l], st);
    if (!rc) rc = alloc((void **)&P->J64[l], sizeof(double) * P->L[l].m->n * P->L[l + 1].m->n);
    if (!rc) rc = interp_matrix<double>(P->L[l].m, P->L[l + 1].m, P->J64[l], st);
  }
  // coarsest level binary64 vectors and solver workspace
  const sem_mesh *cm = P->L.back().m;
  size_t cwb = 0;
  if (!rc) rc = sem_pcg_workspace_bytes(cm, &cwb);
  if (!rc) rc = alloc((void **)&P->cb, sizeof(double) * cm->n_unique);
  if (!rc) rc = alloc((void **)&P->cx, sizeof(double) * cm->n_unique);
  if (!rc && p64) {
    P->L.back().b64 = P->cb;
    P->L.back().x64 = P->cx;
  }
  const bool persistent = cm->K1 && !cm->det_w;  // atomic assembly only: deterministic mode keeps its order
  if (persistent) cwb = std::max(cwb, sem_pcg_n1_workspace_bytes(cm));
  if (!rc) rc = alloc(&P->cws, cwb);
  if (!rc && persistent) {
    rc = alloc((void **)&P->cdinv, sizeof(double) * cm->n_unique);
    if (!rc) rc = sem_jacobi_inv_mode(cm, h1, h2, o->mask_mode ? 0 : 1, P->cdinv, st);
  }
  // outer FCG vectors on the fine level
  const int64_t nU = m->n_unique;
  double **vecs[] = {&P->r, &P->z, &P->zn, &P->p, &P->w};
  for (double **v : vecs)
    if (!rc) rc = alloc((void **)v, sizeof(double) * nU);
  if (!rc) {
    const int npw = std::max(sem_ax_assembled_blocks(m, SEM_PREC_FP64), sem_ax_assembled_blocks(m, SEM_PREC_DF64));
    rc = alloc((void **)&P->pw_part, sizeof(double) * (std::max(npw, 1) + 1));  // + their sum
  }
  cudaError_t e = cudaGetLastError();
  if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (!rc && e != cudaSuccess) rc = sem_cuda_fail(e, "sem_pmg_create");
  if (!rc) rc = check_err(P, st);
  if (rc) {
    free_pmg(P);
    return rc;
  }
  *out = P;
  return SEM_OK;
}

extern "C" int sem_pmg_destroy(sem_pmg *P) {
  free_pmg(P);
  return SEM_OK;
}

extern "C" int sem_pmg_lambda(const sem_pmg *P, int level, double *lambda) {
  if (!P || !lambda || level < 0 || level + 1 >= (int)P->L.size())
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_lambda: bad argument (smoothing levels only)");
  *lambda = P->o.smoother_precision == SEM_PREC_DF64 ? P->L[level].lam64 : (double)P->L[level].lam;
  return SEM_OK;
}

extern "C" int sem_pmg_vcycle(sem_pmg *P, const double *r_g, double *z_g, void *stream) {
  SemRange nvtx_range("sem_pmg_vcycle");
  if (!P || !r_g || !z_g) return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_vcycle: NULL argument");
  cudaStream_t st = as_stream(stream);
  PmgLevel &lv = P->L[0];
  const int64_t n = lv.m->n_unique;
  if (P->o.smoother_precision == SEM_PREC_DF64) {  // binary64 levels: the fine level reads r_g, writes z_g
    double *sb = lv.b64, *sx = lv.x64;
    lv.b64 = const_cast<double *>(r_g);
    lv.x64 = z_g;
    const int rc = vcycle64(P, 0, st);
    lv.b64 = sb;
    lv.x64 = sx;
    if (rc) return rc;
    return check_err(P, st);
  }
  if (P->o.cheb_degree == 2) {
    if (int rc = vcycle2(P, 0, st, r_g, z_g)) return rc;
    return check_err(P, st);
  }
  k_d2f<<<grid_for(n, 256), 256, 0, st>>>(n, r_g, lv.b);
  if (int rc = vcycle(P, 0, st)) return rc;
  k_f2d<<<grid_for(n, 256), 256, 0, st>>>(n, lv.x, z_g);
  SEM_LAUNCH_CHECK("sem_pmg_vcycle");
  return check_err(P, st);
}

extern "C" int sem_pmg_prolong(sem_pmg *P, int level, const double *uc_g, double *uf_g, void *stream) {
  if (!P || !uc_g || !uf_g || level < 0 || level + 1 >= (int)P->L.size())
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_prolong: bad argument");
  cudaStream_t st = as_stream(stream);
  if (P->o.smoother_precision == SEM_PREC_DF64) return prolong64(P, level, uc_g, uf_g, st);
  PmgLevel &f = P->L[level], &c = P->L[level + 1];
  k_d2f<<<grid_for(c.m->n_unique, 256), 256, 0, st>>>(c.m->n_unique, uc_g, c.b);
  if (int rc = prolong_to(P, level, c.b, f.b, st)) return rc;
  k_f2d<<<grid_for(f.m->n_unique, 256), 256, 0, st>>>(f.m->n_unique, f.b, uf_g);
  SEM_LAUNCH_CHECK("sem_pmg_prolong");
  return SEM_OK;
}

extern "C" int sem_pmg_restrict(sem_pmg *P, int level, const double *rf_g, double *rc_g, void *stream) {
  if (!P || !rf_g || !rc_g || level < 0 || level + 1 >= (int)P->L.size())
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_restrict: bad argument");
  cudaStream_t st = as_stream(stream);
  if (P->o.smoother_precision == SEM_PREC_DF64) return restrict64(P, level, rf_g, rc_g, st);
  PmgLevel &f = P->L[level], &c = P->L[level + 1];
  k_d2f<<<grid_for(f.m->n_unique, 256), 256, 0, st>>>(f.m->n_unique, rf_g, f.b);
  if (int rc = restrict_to(P, level, f.b, c.b, st)) return rc;
  k_f2d<<<grid_for(c.m->n_unique, 256), 256, 0, st>>>(c.m->n_unique, c.b, rc_g);
  SEM_LAUNCH_CHECK("sem_pmg_restrict");
  return SEM_OK;
}

extern "C" int sem_pmg_level_apply(sem_pmg *P, int level, const double *u_g, double *w_g, void *stream) {
  if (!P || !u_g || !w_g || u_g == w_g || level < 0 || level + 1 >= (int)P->L.size())
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_level_apply: bad argument (smoothing levels only)");
  cudaStream_t st = as_stream(stream);
  PmgLevel &lv = P->L[level];
  const int64_t n = lv.m->n_unique;
  if (P->o.smoother_precision == SEM_PREC_DF64) {
    SEM_CUDA(cudaMemsetAsync(w_g, 0, sizeof(double) * n, st));
    return ax64(P, level, 1.0, u_g, w_g, st);
  }
  // the level's scratch vectors d (input) and t (output) are free between V-cycles
  k_d2f<<<grid_for(n, 256), 256, 0, st>>>(n, u_g, lv.d);
  SEM_CUDA(cudaMemsetAsync(lv.t, 0, sizeof(float) * n, st));
  if (int rc = ax32(P, level, 1.0f, lv.d, lv.t, st)) return rc;
  k_f2d<<<grid_for(n, 256), 256, 0, st>>>(n, lv.t, w_g);
  SEM_LAUNCH_CHECK("sem_pmg_level_apply");
  return check_err(P, st);
}

extern "C" int sem_pmg_pcg_solve(sem_pmg *P, const double *b_g, double *x_g, const sem_solver_opts *opts,
                                 sem_solve_stats *stats, void *stream) {
  SemRange nvtx_range("sem_pmg_pcg_solve");
  if (!P || !b_g || !x_g || !opts || !stats) return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_pcg_solve: NULL argument");
  if (opts->mask_mode != P->o.mask_mode || (opts->precision != SEM_PREC_FP64 && opts->precision != SEM_PREC_DF64) ||
      !(opts->tol >= 0.0) || opts->maxit < 1 || (opts->initial_guess != 0 && opts->initial_guess != 1))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pmg_pcg_solve: bad options");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = as_stream(stream);
  const sem_mesh *m = P->L[0].m;
  const int64_t n = m->n_unique;
  const unsigned g = grid_for(n, 256);
  int rc;
  stats->iterations = 0;
  stats->status = SEM_OK;
  k_init_fcg<<<g, 256, 0, st>>>(n, b_g, P->o.mask_mode ? nullptr : m->mask, x_g, P->r, opts->initial_guess);
  k_dots<<<kPart, 256, 0, st>>>(n, P->r, P->r, nullptr, nullptr, P->part);
  SEM_LAUNCH_CHECK("fcg init");
  double bb, unused;
  if ((rc = sum_pairs(P->part, &bb, &unused, st))) return rc;
  const double bn = sqrt(bb);
  double rr = bb;
  const bool guess = opts->initial_guess == 1 && bn > 0.0 && std::isfinite(bb);
  if (opts->initial_guess == 1 && !guess) SEM_CUDA(cudaMemsetAsync(x_g, 0, sizeof(double) * n, st));
  if (guess) {  // r = M b - A x: the operator's map leaves r zero on masked nodes
    SEM_CUDA(cudaMemsetAsync(P->w, 0, sizeof(double) * n, st));
    if ((rc = sem_launch_ax_assembled(m, P->h1, P->h2, x_g, P->w, nullptr, opts->precision, st, P->L[0].map)))
      return rc;
    k_sub_from<<<g, 256, 0, st>>>(n, P->w, P->r);
    k_dots<<<kPart, 256, 0, st>>>(n, P->r, P->r, nullptr, nullptr, P->part);
    SEM_LAUNCH_CHECK("fcg initial residual");
    if ((rc = sum_pairs(P->part, &rr, &unused, st))) return rc;
  }
  auto finish = [&](int status, int it, double rr) {
    stats->iterations = it;
    stats->rel_residual = bn > 0 ? sqrt(rr) / bn : 0.0;
    stats->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    stats->status = status;
    if (status == SEM_ERR_NOT_CONVERGED) sem_fail(status, "sem_pmg_pcg_solve: maxit reached");
    if (status == SEM_ERR_BREAKDOWN) sem_fail(status, "sem_pmg_pcg_solve: breakdown");
    return status;
  };
  if (!(bn > 0.0)) return finish(std::isfinite(bb) ? SEM_OK : SEM_ERR_BREAKDOWN, 0, 0.0);
  if (guess) {
    if (!std::isfinite(rr)) return finish(SEM_ERR_BREAKDOWN, 0, rr);
    if (sqrt(rr) <= opts->tol * bn) return finish(SEM_OK, 0, rr);
  }
  if ((rc = sem_pmg_vcycle(P, P->r, P->z, stream))) return rc;
  SEM_CUDA(cudaMemcpyAsync(P->p, P->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  k_dots<<<kPart, 256, 0, st>>>(n, P->r, P->z, nullptr, nullptr, P->part);
  double rz;
  if ((rc = sum_pairs(P->part, &rz, &unused, st))) return rc;
  const int npw = sem_ax_assembled_blocks(m, opts->precision);
  SEM_CUDA(cudaMemsetAsync(P->w, 0, sizeof(double) * n, st));  // later iterations: cleared by k_xpby
  for (int it = 1; it <= opts->maxit; ++it) {
    if ((rc = sem_launch_ax_assembled(m, P->h1, P->h2, P->p, P->w, P->pw_part, opts->precision, st, P->L[0].map)))
      return rc;
    {  // two-level fixed-order sum; P->part (2 kPart doubles) is free until k_dots below
      const int chunk = std::max(1024, (npw + 2 * kPart - 1) / (2 * kPart));
      const int nch = std::max(1, (npw + chunk - 1) / chunk);
      k_sum_chunks<<<nch, 256, 0, st>>>(P->pw_part, npw, chunk, P->part);
      k_sum_fixed<<<1, kSumThreads, 0, st>>>(P->part, nch, P->pw_part + npw);
    }
    SEM_LAUNCH_CHECK("k_sum_fixed");
    double pw = 0.0;
    SEM_CUDA(cudaMemcpyAsync(&pw, P->pw_part + npw, sizeof(double), cudaMemcpyDeviceToHost, st));
    SEM_CUDA(cudaStreamSynchronize(st));
    if (!(pw > 0.0) || !std::isfinite(pw)) return finish(SEM_ERR_BREAKDOWN, it, rr);
    const double alpha = rz / pw;
    k_fcg_update<<<kPart, 256, 0, st>>>(n, alpha, P->p, P->w, x_g, P->r, P->part);
    SEM_LAUNCH_CHECK("fcg update");
    if ((rc = sum_pairs(P->part, &rr, &unused, st))) return rc;
    if (!std::isfinite(rr)) return finish(SEM_ERR_BREAKDOWN, it, rr);
    if (sqrt(rr) <= opts->tol * bn) return finish(SEM_OK, it, rr);
    if (opts->timeout_s > 0.0 &&
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > opts->timeout_s)
      return finish(SEM_ERR_TIMEOUT, it, rr);
    if ((rc = sem_pmg_vcycle(P, P->r, P->zn, stream))) return rc;
    k_dots<<<kPart, 256, 0, st>>>(n, P->r, P->zn, P->r, P->z, P->part);
    double rzn, rzo;
    if ((rc = sum_pairs(P->part, &rzn, &rzo, st))) return rc;
    const double beta = (rzn - rzo) / rz;
    rz = rzn;
    k_xpby<<<g, 256, 0, st>>>(n, P->zn, beta, P->p, P->w);
    SEM_LAUNCH_CHECK("fcg direction");
    std::swap(P->z, P->zn);
  }
  return finish(SEM_ERR_NOT_CONVERGED, opts->maxit, rr);
}
