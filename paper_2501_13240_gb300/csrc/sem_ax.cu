// Matrix-free spectral-element Helmholtz operator (Sec. 2.2): per element,
//   w = h1 [D_r^T D_s^T D_t^T] G [D_r; D_s; D_t] u + h2 B u,
// evaluated by sum factorisation: three 1-D derivative contractions of the
// (N+1)^3 tile, the pointwise multiply by the symmetric 3x3 metric G, and the
// three transposed contractions.
//
// Thread layout: one thread per (i, j) column of an element, looping over k
// (the t-direction contraction stays in registers; r and s go through shared
// memory). ELB elements share a CTA.
#include <algorithm>

#include "sem_internal.h"

namespace {

template <int NP>
struct AxCfg {
  static constexpr int N2 = NP * NP;
  static constexpr int N3 = NP * NP * NP;
  static constexpr int ELB = (N2 >= 256) ? 1 : (256 / N2);  // elements per CTA
  static constexpr int THREADS = N2 * ELB;
  static constexpr int SMEM = (NP * (NP + 1) + 3 * N3 * ELB) * (int)sizeof(double);
};

// FP64 (native DFMA) operator. ASSEMBLED: gather u through l2gm (masked
// local-to-unique map), add results into w with atomics, and accumulate the
// element-local p.w partial sum for the CG step length.
template <int NP, bool ASSEMBLED>
__global__ void __launch_bounds__(AxCfg<NP>::THREADS)
    k_ax_fp64(int64_t E, const double *__restrict__ Dg, const double *__restrict__ G, const double *__restrict__ B,
              double h1, double h2, const double *__restrict__ u, double *__restrict__ w,
              const int32_t *__restrict__ l2gm, double *__restrict__ pw_partial, double *__restrict__ wloc,
              const int *__restrict__ skip, const int32_t *__restrict__ elist) {
  using C = AxCfg<NP>;
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ double smem[];
  double *sD = smem;  // [NP][NP+1]
  const int tid = threadIdx.x;
  const int le = tid / C::N2;
  const int ij = tid - le * C::N2;
  const int i = ij % NP, j = ij / NP;
  double *s_u = smem + NP * (NP + 1) + le * 3 * C::N3;
  double *s_r = s_u + C::N3;
  double *s_s = s_r + C::N3;
  for (int t = tid; t < NP * NP; t += C::THREADS) sD[(t / NP) * (NP + 1) + (t % NP)] = Dg[t];
  double pw = 0.0;
  __syncthreads();
  for (int64_t e0 = (int64_t)blockIdx.x * C::ELB; e0 < E; e0 += (int64_t)gridDim.x * C::ELB) {
    const int64_t ei = e0 + le;  // position in the element list (or the element itself)
    const bool act = ei < E;
    const int64_t e = !act ? 0 : (elist ? (int64_t)elist[ei] : ei);
    double ru[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = i + NP * j + C::N2 * k;
      double v = 0.0;
      if (act) {
        if (ASSEMBLED) {
          const int32_t g = l2gm[e * C::N3 + p];
          v = (g >= 0) ? u[g] : 0.0;
        } else {
          v = u[e * C::N3 + p];
        }
      }
      ru[k] = v;
      s_u[p] = v;
    }
    __syncthreads();
    double rt[NP];
    const double *Ge = G + (act ? e : 0) * 6 * C::N3;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = i + NP * j + C::N2 * k;
      double ur = 0.0, us = 0.0, ut = 0.0;
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        ur = fma(sD[i * (NP + 1) + m], s_u[m + NP * j + C::N2 * k], ur);
        us = fma(sD[j * (NP + 1) + m], s_u[i + NP * m + C::N2 * k], us);
        ut = fma(sD[k * (NP + 1) + m], ru[m], ut);
      }
      double g00 = 0, g01 = 0, g02 = 0, g11 = 0, g12 = 0, g22 = 0;
      if (act) {
        g00 = Ge[p];
        g01 = Ge[C::N3 + p];
        g02 = Ge[2 * C::N3 + p];
        g11 = Ge[3 * C::N3 + p];
        g12 = Ge[4 * C::N3 + p];
        g22 = Ge[5 * C::N3 + p];
      }
      s_r[p] = g00 * ur + g01 * us + g02 * ut;
      s_s[p] = g01 * ur + g11 * us + g12 * ut;
      rt[k] = g02 * ur + g12 * us + g22 * ut;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = i + NP * j + C::N2 * k;
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        acc = fma(sD[m * (NP + 1) + i], s_r[m + NP * j + C::N2 * k], acc);
        acc = fma(sD[m * (NP + 1) + j], s_s[i + NP * m + C::N2 * k], acc);
        acc = fma(sD[m * (NP + 1) + k], rt[m], acc);
      }
      double val = h1 * acc;
      if (h2 != 0.0 && act) val = fma(h2 * B[e * C::N3 + p], ru[k], val);
      if (act) {
        if (ASSEMBLED) {
          const int32_t g = l2gm[e * C::N3 + p];
          if (wloc) wloc[e * C::N3 + p] = (g >= 0) ? val : 0.0;
          else if (g >= 0) atomicAdd(&w[g], val);
          pw = fma(ru[k], val, pw);
        } else {
          w[e * C::N3 + p] = val;
        }
      }
    }
    __syncthreads();
  }
  if (ASSEMBLED && pw_partial != nullptr) {
    // fixed-order CTA sum (the CTA may end in a partial warp, so no full-mask shuffles)
    double *red = smem;  // the tiles are free after the last barrier
    red[tid] = pw;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int t = 0; t < C::THREADS; ++t) s += red[t];
      pw_partial[blockIdx.x] = s;
    }
  }
}

template <int NP, bool ASSEMBLED>
int launch_fp64(const sem_mesh *m, double h1, double h2, const double *u, double *w, double *pw_partial,
                unsigned grid, cudaStream_t st, const int32_t *map, const int *skip, const int32_t *elist = nullptr,
                int64_t nlist = 0) {
  using C = AxCfg<NP>;
  auto kern = k_ax_fp64<NP, ASSEMBLED>;
  if (C::SMEM > 48 * 1024) SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
  double *wloc = (ASSEMBLED && !elist) ? (double *)m->det_w : nullptr;
  kern<<<grid, C::THREADS, C::SMEM, st>>>(elist ? nlist : m->E, m->dD, m->G, m->B, h1, h2, u, w, map, pw_partial,
                                          wloc, skip, elist);
  SEM_LAUNCH_CHECK("k_ax_fp64");
  if (wloc) return sem_launch_gather_add(m, wloc, w, st);
  return SEM_OK;
}

template <int NP>
unsigned ax_grid(const sem_mesh *m, bool assembled) {
  using C = AxCfg<NP>;
  int64_t blocks = (m->E + C::ELB - 1) / C::ELB;
  // the assembled form needs a fixed, mesh-determined grid so that the p.w
  // partial sums are reproducible; cap it at a multiple of the SM count
  if (assembled) blocks = std::min<int64_t>(blocks, 152 * 16);
  return (unsigned)std::max<int64_t>(blocks, 1);
}

template <int NP>
int dispatch_np(const sem_mesh *m, double h1, double h2, const double *u, double *w, double *pw_partial,
                bool assembled, int precision, cudaStream_t st, const int32_t *map, const int *skip) {
  if (precision == SEM_PREC_DF64) return sem_launch_ax_df64(m, h1, h2, u, w, pw_partial, assembled, st, map, skip);
  unsigned grid = ax_grid<NP>(m, assembled);
  if (assembled) return launch_fp64<NP, true>(m, h1, h2, u, w, pw_partial, grid, st, map, skip);
  return launch_fp64<NP, false>(m, h1, h2, u, w, nullptr, grid, st, map, skip);
}

template <int NP>
int dispatch_list_np(const sem_mesh *m, double h1, double h2, const double *u, double *w, int precision,
                     cudaStream_t st, const int32_t *elist, int64_t nlist) {
  if (precision == SEM_PREC_DF64) return sem_launch_ax_df64_list(m, h1, h2, u, w, st, elist, nlist);
  using C = AxCfg<NP>;
  const unsigned grid = (unsigned)std::max<int64_t>(std::min<int64_t>((nlist + C::ELB - 1) / C::ELB, 152 * 16), 1);
  return launch_fp64<NP, true>(m, h1, h2, u, w, nullptr, grid, st, m->l2gm, nullptr, elist, nlist);
}

int dispatch(const sem_mesh *m, double h1, double h2, const double *u, double *w, double *pw_partial, bool assembled,
             int precision, cudaStream_t st, const int32_t *map, const int *skip = nullptr) {
  switch (m->n) {
#define CASE(NPV) \
  case NPV:       \
    return dispatch_np<NPV>(m, h1, h2, u, w, pw_partial, assembled, precision, st, map, skip);
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
#undef CASE
    default:
      return sem_fail(SEM_ERR_INVALID_ARG, "unsupported polynomial order");
  }
}

// Local diagonal of h1 A_L + h2 B: sum_m D_mi^2 G_rr(m,j,k) + ... + 2 D_ii D_jj G_rs + ...
__global__ void k_diag_local(int n, int64_t E, const double *__restrict__ Dg, const double *__restrict__ G,
                             const double *__restrict__ B, double h1, double h2, double *__restrict__ d) {
  const int n3 = n * n * n;
  const int64_t nL = E * n3;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = l / n3;
    const int q = (int)(l - e * n3);
    const int i = q % n, j = (q / n) % n, k = q / (n * n);
    const double *Ge = G + 6 * e * n3;
    double s = 0.0;
    for (int m = 0; m < n; ++m) {
      const double a = Dg[m * n + i], b = Dg[m * n + j], c = Dg[m * n + k];
      s += a * a * Ge[0 * n3 + m + n * (j + n * k)];
      s += b * b * Ge[3 * n3 + i + n * (m + n * k)];
      s += c * c * Ge[5 * n3 + i + n * (j + n * m)];
    }
    const double di = Dg[i * n + i], dj = Dg[j * n + j], dk = Dg[k * n + k];
    s += 2.0 * di * dj * Ge[1 * n3 + q];
    s += 2.0 * di * dk * Ge[2 * n3 + q];
    s += 2.0 * dj * dk * Ge[4 * n3 + q];
    d[l] = h1 * s + h2 * B[l];
  }
}

}  // namespace

int sem_launch_ax_local(const sem_mesh *m, double h1, double h2, const double *u, double *w, int precision,
                        cudaStream_t st) {
  return dispatch(m, h1, h2, u, w, nullptr, false, precision, st, m->l2gm);
}

int sem_launch_ax_assembled(const sem_mesh *m, double h1, double h2, const double *u_g, double *w_g,
                            double *pw_partial, int precision, cudaStream_t st, const int32_t *map, const int *skip) {
  if (m->N == 1 && m->K1)
    return sem_launch_ax_n1(m, h1, h2, u_g, w_g, pw_partial, precision, st, map ? map : m->l2gm, skip);
  return dispatch(m, h1, h2, u_g, w_g, pw_partial, true, precision, st, map ? map : m->l2gm, skip);
}

int sem_launch_ax_assembled_list(const sem_mesh *m, double h1, double h2, const double *u_g, double *w_g,
                                 int precision, cudaStream_t st, const int32_t *elist, int64_t nlist) {
  if (nlist <= 0) return SEM_OK;
  switch (m->n) {  // N = 1 too: the sum-factorised kernels (the element-matrix ones assume the whole mesh)
#define CASE(NPV) \
  case NPV:       \
    return dispatch_list_np<NPV>(m, h1, h2, u_g, w_g, precision, st, elist, nlist);
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
#undef CASE
    default:
      return sem_fail(SEM_ERR_INVALID_ARG, "unsupported polynomial order");
  }
}

int sem_ax_assembled_blocks(const sem_mesh *m, int precision) {
  // element-matrix operator of N = 1 meshes: one element per thread, 128
  // threads per CTA, at most 2 CTAs per SM (few p.w partials to sum)
  if (m->N == 1 && m->K1) return (int)std::max<int64_t>(1, std::min<int64_t>((m->E + 127) / 128, 152 * 2));
  if (precision == SEM_PREC_DF64) return sem_df64_pw_count(m);
  switch (m->n) {
#define CASE(NPV) \
  case NPV:       \
    return (int)ax_grid<NPV>(m, true);
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
#undef CASE
    default:
      return 0;
  }
}

int sem_launch_diag_local(const sem_mesh *m, double h1, double h2, double *dL, cudaStream_t st) {
  k_diag_local<<<grid_for(m->n_local, 256), 256, 0, st>>>(m->n, m->E, m->dD, m->G, m->B, h1, h2, dL);
  SEM_LAUNCH_CHECK("k_diag_local");
  return SEM_OK;
}
