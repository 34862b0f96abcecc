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
// is the p-multigrid coarsest level, whose Jacobi-PCG runs ~100 iterations
// per V-cycle.
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
                 double *__restrict__ pw_partial, double *__restrict__ wloc) {
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
                 double *__restrict__ pw_partial, double *__restrict__ wloc) {
  __shared__ double red[32];
  df::Acc pw = {0.0f, 0.0f};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t gi[8];
    float2 x[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      gi[a] = map[e * 8 + a];
      x[a] = df::from_f64(gi[a] >= 0 ? u[gi[a]] : 0.0);
    }
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
      const double vd = df::to_f64(v.x, v.y);
      if (wloc) wloc[e * 8 + a] = gi[a] >= 0 ? vd : 0.0;
      else if (gi[a] >= 0) atomicAdd(&w[gi[a]], vd);
      if (pw_partial) df::mac(pw, x[a].x, x[a].y, v.x, v.y);
    }
  }
  if (pw_partial) {
    const float2 pn = df::norm(pw);
    const double s = block_pw_sum((double)pn.x + (double)pn.y, red);
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
                     int precision, cudaStream_t st, const int32_t *map) {
  // the grids are those sem_ax_assembled_blocks reports (one p.w partial per CTA)
  const int grid = std::max(sem_ax_assembled_blocks(m, precision), 1);
  double *wloc = (double *)m->det_w;
  if (precision == SEM_PREC_DF64) {
    const float2 h1d = split(h1), h2d = split(h2);
    if (h1 == 1.0 && h2 == 0.0)
      k_ax_n1_df64<false><<<grid, 128, 0, st>>>(m->E, m->K1df, m->Bdf, h1d, h2d, u_g, w_g, map, pw_partial, wloc);
    else
      k_ax_n1_df64<true><<<grid, 128, 0, st>>>(m->E, m->K1df, m->Bdf, h1d, h2d, u_g, w_g, map, pw_partial, wloc);
  } else {
    k_ax_n1_fp64<<<grid, 128, 0, st>>>(m->E, m->K1, m->B, h1, h2, u_g, w_g, map, pw_partial, wloc);
  }
  SEM_LAUNCH_CHECK("k_ax_n1");
  if (wloc) return sem_launch_gather_add(m, wloc, w_g, st);
  return SEM_OK;
}
