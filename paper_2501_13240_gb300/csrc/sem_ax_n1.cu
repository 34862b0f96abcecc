// Linear elements (N = 1, two GLL points per direction): the assembled
// operator of Sec. 2.2 from element matrices instead of sum factorisation.
//
// With two points per direction, sum factorisation does almost no work per
// point and its shared-memory phases dominate; the 8 x 8 element stiffness
//   K[a][b] = sum_q sum_{c,d} (D_c)[q][a] G_cd(q) (D_d)[q][b]
// (the same GLL quadrature, so the same operator) is computed once per mesh
// in binary64 and stored as its 36-entry upper triangle, [entry][element].
// One thread per element then gathers its 8 values, applies K (in binary64,
// or binary64-accurate double-float) and adds h2 B u on the diagonal. This
// is the p-multigrid coarsest level, whose Jacobi-PCG runs ~50 iterations
// per V-cycle (in one persistent launch, below).
#include <algorithm>

#include "sem_df64.cuh"
#include "sem_internal.h"

namespace {

constexpr int kTri = 36;
__host__ __device__ constexpr int tri(int a, int b) {
  return a <= b ? a * 8 - a * (a - 1) / 2 + (b - a) : b * 8 - b * (b - 1) / 2 + (a - b);
}

__global__ void k_n1_matrix(int64_t E, const double *__restrict__ D, const double *__restrict__ G,
                            double *__restrict__ K, float2 *__restrict__ Kdf) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    double Ke[8][8];
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b) Ke[a][b] = 0.0;
    for (int q = 0; q < 8; ++q) {
      double g[6];
      for (int f = 0; f < 6; ++f) g[f] = G[(e * 6 + f) * 8 + q];
      const double Gm[3][3] = {{g[0], g[1], g[2]}, {g[1], g[3], g[4]}, {g[2], g[4], g[5]}};
      for (int c = 0; c < 3; ++c) {
        const int qc = (q >> c) & 1;
        for (int ta = 0; ta < 2; ++ta) {
          const int a = (q & ~(1 << c)) | (ta << c);  // basis a differs from q only along c
          const double ca = D[qc * 2 + ta];
          for (int d = 0; d < 3; ++d) {
            const int qd = (q >> d) & 1;
            for (int tb = 0; tb < 2; ++tb) {
              const int b = (q & ~(1 << d)) | (tb << d);
              Ke[a][b] = fma(ca * Gm[c][d], D[qd * 2 + tb], Ke[a][b]);
            }
          }
        }
      }
    }
    for (int a = 0; a < 8; ++a)
      for (int b = a; b < 8; ++b) {
        const double v = Ke[a][b];
        const float hi = __double2float_rn(v);
        K[(int64_t)tri(a, b) * E + e] = v;
        Kdf[(int64_t)tri(a, b) * E + e] = make_float2(hi, __double2float_rn(v - (double)hi));
      }
  }
}

__device__ __forceinline__ double block_pw_sum(double v, double *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) s += red[t];
  return s;
}

// binary64: w += h1 K u + h2 B u through map; per-CTA p.w partial sums
__global__ void __launch_bounds__(128)
    k_ax_n1_fp64(int64_t E, const double *__restrict__ K, const double *__restrict__ B, double h1, double h2,
                 const double *__restrict__ u, double *__restrict__ w, const int32_t *__restrict__ map,
                 double *__restrict__ pw_partial, double *__restrict__ wloc,
                 const int *__restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  __shared__ double red[32];
  double pw = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t gi[8];
    double x[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      gi[a] = map[e * 8 + a];
      x[a] = gi[a] >= 0 ? u[gi[a]] : 0.0;
    }
    double Kv[kTri];
#pragma unroll
    for (int t = 0; t < kTri; ++t) Kv[t] = K[(int64_t)t * E + e];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      double acc = 0.0;
#pragma unroll
      for (int b = 0; b < 8; ++b) acc = fma(Kv[tri(a, b)], x[b], acc);
      double val = h1 * acc;
      if (h2 != 0.0) val = fma(h2 * B[e * 8 + a], x[a], val);
      if (wloc) wloc[e * 8 + a] = gi[a] >= 0 ? val : 0.0;
      else if (gi[a] >= 0) atomicAdd(&w[gi[a]], val);
      pw = fma(x[a], val, pw);
    }
  }
  if (pw_partial) {
    const double s = block_pw_sum(pw, red);
    if (threadIdx.x == 0) pw_partial[blockIdx.x] = s;
  }
}

// double-float: the same with binary64-accurate compensated dot products
template <bool HELM>
__global__ void __launch_bounds__(128)
    k_ax_n1_df64(int64_t E, const float2 *__restrict__ Kdf, const float2 *__restrict__ Bdf, float2 h1, float2 h2,
                 const double *__restrict__ u, double *__restrict__ w, const int32_t *__restrict__ map,
                 double *__restrict__ pw_partial, double *__restrict__ wloc,
                 const int *__restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  __shared__ double red[32];
  double pw = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t gi[8];
    float2 x[8];
    double uv[8];
    int em = 0;  // the element is computed at the scale 2^-sh of its largest input
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      gi[a] = map[e * 8 + a];
      uv[a] = gi[a] >= 0 ? u[gi[a]] : 0.0;
      em = max(em, df::exp_field(uv[a]));
    }
    const int sh = em - 1023;
#pragma unroll
    for (int a = 0; a < 8; ++a) x[a] = df::from_f64_scaled(uv[a], sh);
    df::Acc pwe = {0.0f, 0.0f};
    float2 Kv[kTri];
#pragma unroll
    for (int t = 0; t < kTri; ++t) Kv[t] = Kdf[(int64_t)t * E + e];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      df::Acc acc = df::mul_first(Kv[tri(a, 0)].x, Kv[tri(a, 0)].y, x[0].x, x[0].y);
#pragma unroll
      for (int b = 1; b < 8; ++b) df::mac(acc, Kv[tri(a, b)].x, Kv[tri(a, b)].y, x[b].x, x[b].y);
      float2 v = df::norm(acc);
      if (HELM) {
        const float2 Bv = Bdf[e * 8 + a];
        const float2 buv = df::norm(df::mul_first(Bv.x, Bv.y, x[a].x, x[a].y));
        df::Acc o = df::mul_first(h1.x, h1.y, v.x, v.y);
        df::mac(o, h2.x, h2.y, buv.x, buv.y);
        v = df::norm(o);
      }
      const double vd = df::to_f64_scaled(v.x, v.y, sh);
      if (wloc) wloc[e * 8 + a] = gi[a] >= 0 ? vd : 0.0;
      else if (gi[a] >= 0) atomicAdd(&w[gi[a]], vd);
      if (pw_partial) df::mac(pwe, x[a].x, x[a].y, v.x, v.y);
    }
    if (pw_partial) {
      const float2 pn = df::norm(pwe);
      pw += df::to_f64_scaled(pn.x, pn.y, 2 * sh);
    }
  }
  if (pw_partial) {
    const double s = block_pw_sum(pw, red);
    if (threadIdx.x == 0) pw_partial[blockIdx.x] = s;
  }
}

float2 split(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

}  // namespace

int sem_n1_prepare(sem_mesh *m, cudaStream_t st) {
  if (m->N != 1) return SEM_OK;
  const size_t cnt = (size_t)kTri * (size_t)std::max<int64_t>(m->E, 1);
  if (cudaMalloc((void **)&m->K1, sizeof(double) * cnt) != cudaSuccess ||
      cudaMalloc((void **)&m->K1df, sizeof(float2) * cnt) != cudaSuccess)
    return sem_fail(SEM_ERR_NOMEM, "sem_mesh_create_box: cudaMalloc(element matrices)");
  k_n1_matrix<<<grid_for(m->E, 128), 128, 0, st>>>(m->E, m->dD, m->G, m->K1, m->K1df);
  SEM_LAUNCH_CHECK("k_n1_matrix");
  return SEM_OK;
}

int sem_launch_ax_n1(const sem_mesh *m, double h1, double h2, const double *u_g, double *w_g, double *pw_partial,
                     int precision, cudaStream_t st, const int32_t *map, const int *skip) {
  // the grids are those sem_ax_assembled_blocks reports (one p.w partial per CTA)
  const int grid = std::max(sem_ax_assembled_blocks(m, precision), 1);
  double *wloc = (double *)m->det_w;
  if (precision == SEM_PREC_DF64) {
    const float2 h1d = split(h1), h2d = split(h2);
    if (h1 == 1.0 && h2 == 0.0)
      k_ax_n1_df64<false><<<grid, 128, 0, st>>>(m->E, m->K1df, m->Bdf, h1d, h2d, u_g, w_g, map, pw_partial, wloc, skip);
    else
      k_ax_n1_df64<true><<<grid, 128, 0, st>>>(m->E, m->K1df, m->Bdf, h1d, h2d, u_g, w_g, map, pw_partial, wloc, skip);
  } else {
    k_ax_n1_fp64<<<grid, 128, 0, st>>>(m->E, m->K1, m->B, h1, h2, u_g, w_g, map, pw_partial, wloc, skip);
  }
  SEM_LAUNCH_CHECK("k_ax_n1");
  if (wloc) return sem_launch_gather_add(m, wloc, w_g, st);
  return SEM_OK;
}

// ---------------------------------------------------------------- persistent coarse Jacobi-PCG
// The p-multigrid coarsest level (N = 1) is solved by ~50 Jacobi-PCG
// iterations per V-cycle, each a few microseconds of work; as separate
// launches with host checks its cost is launch and synchronisation latency.
// Here the whole solve is one cooperative launch: the CTAs meet at grid
// barriers (three per iteration) built on a global counter, every wait
// bounded (on timeout an error flag ends the kernel), reductions in a fixed
// order that every CTA repeats, so all CTAs take the same decisions. Same
// algorithm as sem_pcg_solve: x0 = 0, the system scaled by a power of two
// with ||b|| ~ 1, stop at the first ||r|| <= tol ||b||, breakdown on
// p.Ap <= 0 or a non-finite scalar; double-float operator, binary64 vectors.
namespace {

struct GridBar {
  unsigned count, gen;
  int err, pad;
};

__device__ bool grid_sync(GridBar *gb, unsigned nblocks, unsigned spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = &gb->gen;
    const unsigned g0 = *vgen;
    __threadfence();  // this CTA's writes before its arrival
    bool ok = true;
    if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      for (unsigned it = 0; *vgen == g0; ++it) {
        if (it >= spin_limit) {
          ok = false;
          atomicExch(&gb->err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();  // the other CTAs' writes after the barrier
    s_ok = ok && *(volatile int *)&gb->err == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ double block_sum_d(double v, double *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int t = 0; t < (int)(blockDim.x >> 5); ++t) s += red[t];  // every thread, same order
  return s;
}

// sum of slot `q` of the per-CTA partials, in the same order in every CTA
__device__ __forceinline__ double sum_parts(const double *part, unsigned nb, int q, double *red) {
  double s = 0.0;
  for (unsigned i = threadIdx.x; i < nb; i += blockDim.x) s += ((volatile const double *)part)[4 * i + q];
  return block_sum_d(s, red);
}

struct CoarseArgs {
  int64_t E, nU;
  const float2 *Kdf, *Bdf;
  float2 h1, h2;
  const int32_t *map;
  const double *dinv, *b;
  double *x, *r, *p, *w, *part;
  GridBar *bar;
  int *out_status, *out_iters;
  double *out_rel;
  double tol;
  int maxit;
  unsigned spin_limit;  // polls of a grid-barrier wait before it gives up
};

// w += h1 K p (+ h2 B p) over this thread's elements; returns its p.w contribution
template <bool HELM>
__device__ __forceinline__ double n1_apply(const CoarseArgs &a, int64_t e0, int64_t estride) {
  df::Acc pw = {0.0f, 0.0f};
  for (int64_t e = e0; e < a.E; e += estride) {
    int32_t gi[8];
    float2 x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      gi[q] = a.map[e * 8 + q];
      x[q] = df::from_f64(gi[q] >= 0 ? __ldcg(a.p + gi[q]) : 0.0);  // p of other CTAs: not from L1
    }
    float2 Kv[kTri];
#pragma unroll
    for (int t = 0; t < kTri; ++t) Kv[t] = a.Kdf[(int64_t)t * a.E + e];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      df::Acc acc = df::mul_first(Kv[tri(q, 0)].x, Kv[tri(q, 0)].y, x[0].x, x[0].y);
#pragma unroll
      for (int s = 1; s < 8; ++s) df::mac(acc, Kv[tri(q, s)].x, Kv[tri(q, s)].y, x[s].x, x[s].y);
      float2 v = df::norm(acc);
      if (HELM) {
        const float2 Bv = a.Bdf[e * 8 + q];
        const float2 buv = df::norm(df::mul_first(Bv.x, Bv.y, x[q].x, x[q].y));
        df::Acc o = df::mul_first(a.h1.x, a.h1.y, v.x, v.y);
        df::mac(o, a.h2.x, a.h2.y, buv.x, buv.y);
        v = df::norm(o);
      }
      if (gi[q] >= 0) atomicAdd(&a.w[gi[q]], df::to_f64(v.x, v.y));
      df::mac(pw, x[q].x, x[q].y, v.x, v.y);
    }
  }
  const float2 pn = df::norm(pw);
  return (double)pn.x + (double)pn.y;
}

template <bool HELM>
__global__ void __launch_bounds__(256, 2) k_pcg_n1(CoarseArgs a) {
  __shared__ double red[32];
  const unsigned nb = gridDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
  double *mine = a.part + 4 * (int64_t)blockIdx.x;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  // ||b||^2
  double s = 0.0;
  for (int64_t g = t0; g < a.nU; g += nt) s = fma(a.b[g], a.b[g], s);
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) mine[0] = s;
  if (!grid_sync(a.bar, nb, a.spin_limit)) return;
  const double bb = sum_parts(a.part, nb, 0, red);
  const double bnorm = sqrt(bb);
  if (!(bnorm > 0.0) || !isfinite(bb)) {
    for (int64_t g = t0; g < a.nU; g += nt) a.x[g] = 0.0;
    if (lead) {
      *a.out_status = isfinite(bb) ? SEM_OK : SEM_ERR_BREAKDOWN;
      *a.out_iters = 0;
      *a.out_rel = 0.0;
    }
    return;
  }
  const double scale = ldexp(1.0, ilogb(bnorm)), inv = 1.0 / scale;  // exact powers of two
  // r = b / scale, x = 0, w = 0, p = z = D^{-1} r
  s = 0.0;
  for (int64_t g = t0; g < a.nU; g += nt) {
    const double rv = a.b[g] * inv, zv = a.dinv[g] * rv;
    a.r[g] = rv;
    a.x[g] = 0.0;
    a.w[g] = 0.0;
    a.p[g] = zv;
    s = fma(rv, zv, s);
  }
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) mine[1] = s;
  if (!grid_sync(a.bar, nb, a.spin_limit)) return;
  double rz = sum_parts(a.part, nb, 1, red), rr = bb * inv * inv;
  const double thresh = a.tol * bnorm * inv;
  int status = SEM_ERR_NOT_CONVERGED, it = 0;
  while (it < a.maxit) {
    ++it;
    s = n1_apply<HELM>(a, t0, nt);  // w = A p
    s = block_sum_d(s, red);
    if (threadIdx.x == 0) mine[2] = s;
    if (!grid_sync(a.bar, nb, a.spin_limit)) return;
    const double pw = sum_parts(a.part, nb, 2, red);
    if (!(pw > 0.0) || !isfinite(pw)) {
      status = SEM_ERR_BREAKDOWN;
      break;
    }
    const double alpha = rz / pw;
    double sz = 0.0, sr = 0.0;
    for (int64_t g = t0; g < a.nU; g += nt) {
      const double rv = fma(-alpha, __ldcg(a.w + g), a.r[g]);  // w was summed by atomics in L2
      a.x[g] = fma(alpha, a.p[g], a.x[g]);
      a.r[g] = rv;
      a.w[g] = 0.0;
      sz = fma(rv, a.dinv[g] * rv, sz);
      sr = fma(rv, rv, sr);
    }
    sz = block_sum_d(sz, red);
    sr = block_sum_d(sr, red);
    if (threadIdx.x == 0) {
      mine[3] = sz;
      mine[0] = sr;
    }
    if (!grid_sync(a.bar, nb, a.spin_limit)) return;
    const double rzn = sum_parts(a.part, nb, 3, red);
    rr = sum_parts(a.part, nb, 0, red);
    if (isfinite(rr) && sqrt(rr) <= thresh) {
      status = SEM_OK;
      break;
    }
    if (!isfinite(rr) || !isfinite(rzn)) {
      status = SEM_ERR_BREAKDOWN;
      break;
    }
    const double beta = rzn / rz;
    rz = rzn;
    for (int64_t g = t0; g < a.nU; g += nt) a.p[g] = fma(beta, a.p[g], a.dinv[g] * a.r[g]);
    if (!grid_sync(a.bar, nb, a.spin_limit)) return;
  }
  for (int64_t g = t0; g < a.nU; g += nt) a.x[g] *= scale;
  if (lead) {
    *a.out_status = status;
    *a.out_iters = it;
    *a.out_rel = sqrt(rr) / (bnorm * inv);
  }
}

}  // namespace

size_t sem_pcg_n1_workspace_bytes(const sem_mesh *m) {
  return sizeof(double) * (3 * (size_t)m->n_unique + 4 * 152 * 8) + 256;
}

// Solve (h1 A + h2 B) x = b on an N = 1 mesh (b: masked as the operator's
// map); `work` holds sem_pcg_n1_workspace_bytes(m) bytes, dinv the Jacobi
// inverse. Returns the status of the solve; *iters and *rel when not NULL.
int sem_pcg_n1_persistent(const sem_mesh *m, double h1, double h2, const double *b, double *x, const double *dinv,
                          const int32_t *map, double tol, int maxit, void *work, int *iters, double *rel,
                          cudaStream_t st) {
  if (m->N != 1 || !m->K1df) return sem_fail(SEM_ERR_INVALID_ARG, "coarse solve: not an N = 1 mesh");
  const bool helm = !(h1 == 1.0 && h2 == 0.0);
  auto kern = helm ? k_pcg_n1<true> : k_pcg_n1<false>;
  int per_sm = 0, nsm = 0, coop = 0;
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0));
  SEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
  SEM_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, m->device));
  if (!coop || per_sm < 1) return sem_fail(SEM_ERR_CUDA, "coarse solve: cooperative launch unavailable");
  const unsigned nb = (unsigned)std::min<int64_t>(std::min(per_sm, 8) * (int64_t)std::min(nsm, 152),
                                                  std::max<int64_t>(1, (m->n_unique + 255) / 256));
  char *w8 = reinterpret_cast<char *>(work);
  CoarseArgs a;
  a.E = m->E;
  a.nU = m->n_unique;
  a.Kdf = m->K1df;
  a.Bdf = m->Bdf;
  a.h1 = split(h1);
  a.h2 = split(h2);
  a.map = map;
  a.dinv = dinv;
  a.b = b;
  a.x = x;
  a.r = reinterpret_cast<double *>(w8);
  a.p = a.r + m->n_unique;
  a.w = a.p + m->n_unique;
  a.part = a.w + m->n_unique;                                    // 4 doubles per CTA
  GridBar *bar = reinterpret_cast<GridBar *>(a.part + 4 * 152 * 8);
  int *ires = reinterpret_cast<int *>(bar + 1);
  a.bar = bar;
  a.out_status = ires;
  a.out_iters = ires + 1;
  a.out_rel = reinterpret_cast<double *>(ires + 2);
  a.tol = tol;
  a.maxit = maxit;
  a.spin_limit = sem_grid_wait_limit();
  SEM_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBar), st));
  void *args[] = {&a};
  SEM_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3(nb), dim3(256), args, 0, st));
  struct {
    GridBar bar;
    int status, iters;
    double rel;
  } h;
  SEM_CUDA(cudaMemcpyAsync(&h, bar, sizeof(h), cudaMemcpyDeviceToHost, st));
  SEM_CUDA(cudaStreamSynchronize(st));
  if (h.bar.err) return sem_fail(SEM_ERR_CUDA, "coarse solve: a grid barrier wait exceeded its limit");
  if (iters) *iters = h.iters;
  if (rel) *rel = h.rel;
  if (h.status == SEM_ERR_BREAKDOWN) return sem_fail(SEM_ERR_BREAKDOWN, "coarse solve: breakdown");
  if (h.status == SEM_ERR_NOT_CONVERGED) return sem_fail(SEM_ERR_NOT_CONVERGED, "coarse solve: maxit reached");
  return SEM_OK;
}
