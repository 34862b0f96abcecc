// Mesh and GLL set-up: node coordinates, geometric factors (chain rule,
// Sec. 2.2), lattice local-to-unique map, Dirichlet mask and the
// gather-scatter (Q Q^T) tables. All per-node work runs in kernels.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "sem_internal.h"

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;

int sem_fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

int sem_cuda_fail(cudaError_t e, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return (e == cudaErrorMemoryAllocation) ? SEM_ERR_NOMEM : SEM_ERR_CUDA;
}

extern "C" const char *sem_last_error(void) { return g_last_error.c_str(); }
extern "C" const char *sem_version(void) { return "semgb 0.1 (sm_103a)"; }

// ---------------------------------------------------------------- bounded device waits
static std::atomic<unsigned> g_grid_wait_limit{1u << 24};

unsigned sem_grid_wait_limit() { return g_grid_wait_limit.load(std::memory_order_relaxed); }

extern "C" int sem_set_grid_wait_limit(unsigned polls, unsigned *previous) {
  const unsigned old = g_grid_wait_limit.exchange(polls == 0 ? (1u << 24) : polls);
  if (previous) *previous = old;
  return SEM_OK;
}

// ---------------------------------------------------------------- GLL
// Interior GLL nodes are the zeros of (1 - x^2) P_N'(x) = N (P_{N-1}(x) - x P_N(x)).
// Newton's method on q(x) = P_{N-1}(x) - x P_N(x), q'(x) = -(N+1) P_N(x), from the
// Chebyshev-Gauss-Lobatto points, in long double.
static void leg_pair(int N, long double x, long double &pn, long double &pnm1) {
  long double a = 1.0L, b = x;  // P_0, P_1
  if (N == 0) { pn = 1.0L; pnm1 = 0.0L; return; }
  for (int k = 1; k < N; ++k) {
    long double c = ((2.0L * k + 1.0L) * x * b - k * a) / (k + 1.0L);
    a = b;
    b = c;
  }
  pn = b;
  pnm1 = a;
}

int sem_gll_host(int N, double *xi, double *rho, double *D) {
  if (N < 1 || N > SEM_MAXN || !xi || !rho || !D)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_gll: N must be in [1, 10] and arrays non-NULL");
  const int n = N + 1;
  long double x[SEM_MAXNP], PN[SEM_MAXNP];
  const long double PI = 3.14159265358979323846264338327950288L;
  for (int i = 0; i < n; ++i) {
    long double t = -cosl(PI * (long double)i / (long double)N);
    if (i != 0 && i != N) {
      for (int it = 0; it < 60; ++it) {
        long double pn, pm;
        leg_pair(N, t, pn, pm);
        long double q = pm - t * pn;
        long double dq = -(N + 1.0L) * pn;
        long double dt = q / dq;
        t -= dt;
        if (fabsl(dt) <= 1e-20L) break;
      }
    }
    x[i] = t;
  }
  x[0] = -1.0L;
  x[N] = 1.0L;
  for (int i = 0; i < n / 2; ++i) {  // symmetric pairs
    long double s = 0.5L * (x[N - i] - x[i]);
    x[i] = -s;
    x[N - i] = s;
  }
  if ((N & 1) == 0) x[N / 2] = 0.0L;
  for (int i = 0; i < n; ++i) {
    long double pm;
    leg_pair(N, x[i], PN[i], pm);
    xi[i] = (double)x[i];
    rho[i] = (double)(2.0L / ((long double)N * (N + 1) * PN[i] * PN[i]));
  }
  const long double dcorner = (long double)N * (N + 1) / 4.0L;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      long double v = 0.0L;
      if (i != j) v = PN[i] / (PN[j] * (x[i] - x[j]));
      else if (i == 0) v = -dcorner;
      else if (i == N) v = dcorner;
      D[i * n + j] = (double)v;
    }
  return SEM_OK;
}

extern "C" int sem_gll(int N, double *xi, double *rho, double *D) { return sem_gll_host(N, xi, rho, D); }

// ---------------------------------------------------------------- kernels
struct BoxParams {
  int nel[3];
  int N, n;
  double L[3];
  double s;  // z stretch
  double amp;
  double kappa[9];
  double phi[3];
  double xi[SEM_MAXNP];
  int periodic[3];
  int dirichlet[6];
  int64_t nd[3];  // unique lattice extent per direction (z: of the slab)
  // a slab of whole element planes: elements e_off.. of the box, lattice
  // planes from k_off; wrapz: z is periodic and the slab is the whole box
  int64_t e_off, k_off;
  int wrapz;
};

__device__ __forceinline__ double iface(const BoxParams &p, int d, int k) {
  if (d == 2 && p.s > 0.0) return 0.5 * p.L[2] * (1.0 + tanh(p.s * (2.0 * k / p.nel[2] - 1.0)) / tanh(p.s));
  return p.L[d] * (double)k / (double)p.nel[d];
}

__global__ void k_coords(BoxParams p, int64_t nL, double *X, double *Y, double *Z) {
  const int n = p.n, n3 = n * n * n;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t el = l / n3;
    int q = (int)(l - el * n3);
    const int64_t e = el + p.e_off;  // element of the whole box
    int loc[3] = {q % n, (q / n) % n, q / (n * n)};
    int64_t ex = e % p.nel[0];
    int64_t ey = (e / p.nel[0]) % p.nel[1];
    int64_t ez = e / ((int64_t)p.nel[0] * p.nel[1]);
    int eidx[3] = {(int)ex, (int)ey, (int)ez};
    double x[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double a = iface(p, d, eidx[d]), b = iface(p, d, eidx[d] + 1);
      double t = p.xi[loc[d]];
      x[d] = a * (0.5 * (1.0 - t)) + b * (0.5 * (1.0 + t));
    }
    double o[3] = {x[0], x[1], x[2]};
    if (p.amp != 0.0) {
      const double PI = 3.14159265358979323846;
      double xh = x[0] / p.L[0], yh = x[1] / p.L[1], zh = x[2] / p.L[2];
      double bump = sin(PI * xh) * sin(PI * yh) * sin(PI * zh);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double arg = 2.0 * PI * (p.kappa[3 * c] * xh + p.kappa[3 * c + 1] * yh + p.kappa[3 * c + 2] * zh) + p.phi[c];
        o[c] = x[c] + p.amp * (p.L[c] / p.nel[c]) * bump * cos(arg);
      }
    }
    X[l] = o[0];
    Y[l] = o[1];
    Z[l] = o[2];
  }
}

// Split a binary64 into hi + lo binary32 (hi = RN(x), lo = RN(x - hi)).
__device__ __forceinline__ float2 split_df(double v) {
  float hi = __double2float_rn(v);
  float lo = __double2float_rn(v - (double)hi);
  return make_float2(hi, lo);
}

// One CTA per element: Jacobian by D applied to the node coordinates, its
// inverse by cofactors, G_ab = w |J| sum_c dr_a/dx_c dr_b/dx_c, B = w |J|.
__global__ void k_geom(int n, int64_t E, const double *__restrict__ Dg, const double *__restrict__ rho,
                       const double *__restrict__ X, const double *__restrict__ Y, const double *__restrict__ Z,
                       double *__restrict__ G, float2 *__restrict__ Gdf, double *__restrict__ B,
                       float2 *__restrict__ Bdf, double *__restrict__ detmin_e) {
  __shared__ double sD[SEM_MAXNP * SEM_MAXNP];
  __shared__ double red[32];
  const int n3 = n * n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) sD[t] = Dg[t];
  __syncthreads();
  for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
    const int64_t base = e * n3;
    double dmin = INFINITY;
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
      const int i = q % n, j = (q / n) % n, k = q / (n * n);
      double J[3][3];
      const double *xc[3] = {X + base, Y + base, Z + base};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double a = 0.0, b = 0.0, d = 0.0;
        for (int m = 0; m < n; ++m) {
          a = fma(sD[i * n + m], xc[c][m + n * (j + n * k)], a);
          b = fma(sD[j * n + m], xc[c][i + n * (m + n * k)], b);
          d = fma(sD[k * n + m], xc[c][i + n * (j + n * m)], d);
        }
        J[c][0] = a;
        J[c][1] = b;
        J[c][2] = d;
      }
      // cofactor matrix C[c][a]; inverse R[a][c] = C[c][a] / det
      double C00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      double C01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      double C02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      double C10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
      double C11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
      double C12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
      double C20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
      double C21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
      double C22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      double det = J[0][0] * C00 + J[0][1] * C01 + J[0][2] * C02;
      dmin = fmin(dmin, det);
      double inv = 1.0 / det;
      // R[a][c] = C[c][a] * inv
      double R[3][3] = {{C00 * inv, C10 * inv, C20 * inv}, {C01 * inv, C11 * inv, C21 * inv},
                        {C02 * inv, C12 * inv, C22 * inv}};
      double w = rho[i] * rho[j] * rho[k] * det;
      const int fa[6] = {0, 0, 0, 1, 1, 2}, fb[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        double g = w * (R[fa[f]][0] * R[fb[f]][0] + R[fa[f]][1] * R[fb[f]][1] + R[fa[f]][2] * R[fb[f]][2]);
        G[(6 * e + f) * n3 + q] = g;
        Gdf[(6 * e + f) * n3 + q] = split_df(g);
      }
      B[base + q] = w;
      Bdf[base + q] = split_df(w);
    }
    // block min of det J
    for (int off = 16; off > 0; off >>= 1) dmin = fmin(dmin, __shfl_xor_sync(0xffffffffu, dmin, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dmin;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = red[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = fmin(v, red[w]);
      detmin_e[e] = v;
    }
    __syncthreads();
  }
}

__global__ void k_l2g(BoxParams p, int64_t nL, int32_t *l2g) {
  const int n = p.n, n3 = n * n * n, N = p.N;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = l / n3;
    int q = (int)(l - e * n3);
    e += p.e_off;
    int64_t ex = e % p.nel[0], ey = (e / p.nel[0]) % p.nel[1], ez = e / ((int64_t)p.nel[0] * p.nel[1]);
    int64_t I = ex * N + q % n, J = ey * N + (q / n) % n, K = ez * N + q / (n * n);
    if (p.periodic[0] && I == (int64_t)p.nel[0] * N) I = 0;
    if (p.periodic[1] && J == (int64_t)p.nel[1] * N) J = 0;
    if (p.wrapz && K == (int64_t)p.nel[2] * N) K = 0;
    l2g[l] = (int32_t)(I + p.nd[0] * (J + p.nd[1] * (K - p.k_off)));
  }
}

__global__ void k_mask(BoxParams p, int64_t nU, uint8_t *mask) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nU; g += (int64_t)gridDim.x * blockDim.x) {
    // lattice indices in the whole box (z offset by the slab's first plane)
    int64_t idx[3] = {g % p.nd[0], (g / p.nd[0]) % p.nd[1], g / (p.nd[0] * p.nd[1]) + p.k_off};
    const int64_t top[3] = {p.nd[0] - 1, p.nd[1] - 1, (int64_t)p.nel[2] * p.N};
    uint8_t m = 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (p.periodic[d]) continue;
      if (p.dirichlet[2 * d] && idx[d] == 0) m = 0;
      if (p.dirichlet[2 * d + 1] && idx[d] == top[d]) m = 0;
    }
    mask[g] = m;
  }
}

__global__ void k_l2gm(int64_t nL, const int32_t *l2g, const uint8_t *mask, int32_t *l2gm) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    int32_t g = l2g[l];
    l2gm[l] = mask[g] ? g : -1;
  }
}

__global__ void k_count(int64_t nL, const int32_t *l2g, int32_t *cnt) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[l2g[l]], 1);
}

// Exclusive scan, first pass: each block scans SCAN_TILE consecutive values.
#define SCAN_THREADS 1024
#define SCAN_PER 4
#define SCAN_TILE (SCAN_THREADS * SCAN_PER)
__global__ void k_scan_tile(const int32_t *in, int32_t *out, int64_t n, int32_t *tile_sums) {
  __shared__ int32_t warp_tot[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER;
  int32_t v[SCAN_PER];
  int32_t s = 0;
#pragma unroll
  for (int t = 0; t < SCAN_PER; ++t) {
    v[t] = (base + t < n) ? in[base + t] : 0;
    s += v[t];
  }
  // inclusive warp scan of per-thread sums
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t inc = s;
  for (int off = 1; off < 32; off <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += y;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int32_t w = warp_tot[lane];
    for (int off = 1; off < 32; off <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    warp_tot[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  int32_t run = inc - s + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
  for (int t = 0; t < SCAN_PER; ++t) {
    if (base + t < n) out[base + t] = run;
    run += v[t];
  }
  if (threadIdx.x == SCAN_THREADS - 1) tile_sums[blockIdx.x] = warp_tot[31];
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *tile_off) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] += tile_off[i / SCAN_TILE];
}

__global__ void k_fill(int64_t nL, const int32_t *l2g, int32_t *pos, int32_t *perm) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    int32_t k = atomicAdd(&pos[l2g[l]], 1);
    perm[k] = (int32_t)l;
  }
}

// Sort each unique node's list of local copies (ascending) so that summation
// order -- and hence every gather-scatter result -- is deterministic.
__global__ void k_sort_segments(int64_t nU, const int32_t *off, int32_t *perm, double *mult) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nU; g += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = off[g], b = off[g + 1];
    for (int32_t s = a + 1; s < b; ++s) {
      int32_t v = perm[s];
      int32_t t = s - 1;
      while (t >= a && perm[t] > v) {
        perm[t + 1] = perm[t];
        --t;
      }
      perm[t + 1] = v;
    }
    mult[g] = (double)(b - a);
  }
}

// ---------------------------------------------------------------- host
static void free_mesh(sem_mesh *m) {
  if (!m) return;
  void *ptrs[] = {m->X,    m->Y,    m->Z,      m->G,      m->Gdf,  m->B,     m->Bdf, m->l2g,
                  m->l2gm, m->mask, m->mult,   m->gs_off, m->gs_perm, m->dD, m->det_w, m->K1, m->K1df,
                  m->Gt,   m->Mt};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete m;
}

template <typename T>
static int dalloc(T **p, size_t count, const char *what) {
  cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    *p = nullptr;
    return sem_cuda_fail(e, what);
  }
  return SEM_OK;
}

static int build_gs_tables(sem_mesh *m, cudaStream_t st) {
  const int64_t nL = m->n_local, nU = m->n_unique;
  int rc;
  int32_t *cnt = nullptr, *pos = nullptr, *tiles = nullptr;
  const int64_t ntile = (nU + 1 + SCAN_TILE - 1) / SCAN_TILE;
  if ((rc = dalloc(&m->gs_off, nU + 1, "cudaMalloc(gs_off)")) ||
      (rc = dalloc(&m->gs_perm, nL, "cudaMalloc(gs_perm)")) || (rc = dalloc(&m->mult, nU, "cudaMalloc(mult)")) ||
      (rc = dalloc(&cnt, nU + 1, "cudaMalloc(count)")) || (rc = dalloc(&pos, nU + 1, "cudaMalloc(pos)")) ||
      (rc = dalloc(&tiles, ntile, "cudaMalloc(tiles)"))) {
    cudaFree(cnt);
    cudaFree(pos);
    cudaFree(tiles);
    return rc;
  }
  auto cleanup = [&]() {
    cudaFree(cnt);
    cudaFree(pos);
    cudaFree(tiles);
  };
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nU + 1), st);
  k_count<<<grid_for(nL, 256), 256, 0, st>>>(nL, m->l2g, cnt);
  k_scan_tile<<<(unsigned)ntile, SCAN_THREADS, 0, st>>>(cnt, m->gs_off, nU + 1, tiles);
  std::vector<int32_t> h(ntile);
  cudaError_t e = cudaMemcpyAsync(h.data(), tiles, sizeof(int32_t) * ntile, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cleanup();
    return sem_cuda_fail(e, "gs table scan");
  }
  int64_t run = 0;
  for (int64_t t = 0; t < ntile; ++t) {
    int64_t v = h[t];
    h[t] = (int32_t)run;
    run += v;
  }
  if (run != nL) {
    cleanup();
    return sem_fail(SEM_ERR_CUDA, "gs table scan: total count mismatch");
  }
  cudaMemcpyAsync(tiles, h.data(), sizeof(int32_t) * ntile, cudaMemcpyHostToDevice, st);
  k_scan_add<<<grid_for(nU + 1, 256), 256, 0, st>>>(m->gs_off, nU + 1, tiles);
  cudaMemcpyAsync(pos, m->gs_off, sizeof(int32_t) * (nU + 1), cudaMemcpyDeviceToDevice, st);
  k_fill<<<grid_for(nL, 256), 256, 0, st>>>(nL, m->l2g, pos, m->gs_perm);
  k_sort_segments<<<grid_for(nU, 256), 256, 0, st>>>(nU, m->gs_off, m->gs_perm, m->mult);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return sem_cuda_fail(e, "gs table build");
  return SEM_OK;
}

extern "C" int sem_mesh_create_box(const sem_box_desc *d, void *stream, sem_mesh **out) {
  return sem_mesh_create_slab(d, 0, -1, stream, out);
}

// The box, or the slab of its element planes [p0, p1) (p1 < 0: the whole box):
// the slab's elements in box order, its own unique numbering of lattice
// planes p0 N .. p1 N (no periodic wrap in z unless it is the whole box).
int sem_mesh_create_slab(const sem_box_desc *d, int p0, int p1, void *stream, sem_mesh **out) {
  SemRange nvtx_range("sem_mesh_create_box");
  if (!d || !out) return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_create_box: NULL argument");
  *out = nullptr;
  if (d->N < 1 || d->N > SEM_MAXN) return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_create_box: N must be in [1, 10]");
  if (d->nelx < 1 || d->nely < 1 || d->nelz < 1)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_create_box: element counts must be >= 1");
  if (!(d->Lx > 0 && d->Ly > 0 && d->Lz > 0)) return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_create_box: lengths must be > 0");
  if (d->z_stretch < 0 || !std::isfinite(d->z_stretch) || !std::isfinite(d->deform_amp))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_create_box: bad stretch or deformation amplitude");
  for (int c = 0; c < 3; ++c)
    if (d->periodic[c] && (c == 0 ? d->nelx : c == 1 ? d->nely : d->nelz) < 2)
      return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_create_box: a periodic direction needs >= 2 elements");
  const int n = d->N + 1;
  if (p1 < 0) {
    p0 = 0;
    p1 = d->nelz;
  }
  if (p0 < 0 || p1 > d->nelz || p0 >= p1) return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_create_box: bad slab");
  const bool whole = (p0 == 0 && p1 == d->nelz);
  const int64_t plane = (int64_t)d->nelx * d->nely;
  const int64_t E = plane * (p1 - p0);
  const int64_t nL = E * n * n * n;
  if (nL > 2147483647LL) return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_create_box: more than 2^31-1 local nodes");
  cudaStream_t st = as_stream(stream);

  sem_mesh *m = new sem_mesh();
  m->nel[0] = d->nelx;
  m->nel[1] = d->nely;
  m->nel[2] = p1 - p0;
  m->slab = whole ? 0 : 1;
  m->slab_p0 = p0;
  m->N = d->N;
  m->n = n;
  m->n3 = n * n * n;
  m->E = E;
  m->n_local = nL;
  for (int c = 0; c < 3; ++c) m->periodic[c] = d->periodic[c] ? 1 : 0;
  for (int f = 0; f < 6; ++f) m->dirichlet[f] = d->dirichlet[f] ? 1 : 0;
  m->L[0] = d->Lx;
  m->L[1] = d->Ly;
  m->L[2] = d->Lz;
  m->desc = *d;
  cudaGetDevice(&m->device);
  sem_gll_host(d->N, m->xi, m->rho, m->D);

  BoxParams p;
  memset(&p, 0, sizeof(p));
  const int nel_box[3] = {d->nelx, d->nely, d->nelz};
  for (int c = 0; c < 3; ++c) {
    p.nel[c] = nel_box[c];
    p.L[c] = m->L[c];
    p.periodic[c] = m->periodic[c];
    p.nd[c] = (int64_t)nel_box[c] * d->N + (m->periodic[c] ? 0 : 1);
  }
  p.e_off = plane * p0;
  p.k_off = (int64_t)p0 * d->N;
  p.wrapz = (m->periodic[2] && whole) ? 1 : 0;
  if (!whole) p.nd[2] = (int64_t)(p1 - p0) * d->N + 1;
  for (int f = 0; f < 6; ++f) p.dirichlet[f] = m->dirichlet[f];
  p.N = d->N;
  p.n = n;
  p.s = d->z_stretch;
  p.amp = d->deform_amp;
  for (int t = 0; t < 9; ++t) p.kappa[t] = d->kappa[t];
  for (int t = 0; t < 3; ++t) p.phi[t] = d->phi[t];
  for (int t = 0; t < n; ++t) p.xi[t] = m->xi[t];
  m->n_unique = p.nd[0] * p.nd[1] * p.nd[2];

  int rc;
  double *rho_d = nullptr, *detmin_e = nullptr;
  if ((rc = dalloc(&m->X, nL, "cudaMalloc(X)")) || (rc = dalloc(&m->Y, nL, "cudaMalloc(Y)")) ||
      (rc = dalloc(&m->Z, nL, "cudaMalloc(Z)")) || (rc = dalloc(&m->G, 6 * nL, "cudaMalloc(G)")) ||
      (rc = dalloc(&m->Gdf, 6 * nL, "cudaMalloc(Gdf)")) || (rc = dalloc(&m->B, nL, "cudaMalloc(B)")) ||
      (rc = dalloc(&m->Bdf, nL, "cudaMalloc(Bdf)")) ||
      (rc = dalloc(&m->l2g, nL, "cudaMalloc(l2g)")) || (rc = dalloc(&m->l2gm, nL, "cudaMalloc(l2gm)")) ||
      (rc = dalloc(&m->mask, m->n_unique, "cudaMalloc(mask)")) || (rc = dalloc(&m->dD, n * n, "cudaMalloc(D)")) ||
      (rc = dalloc(&rho_d, n, "cudaMalloc(rho)")) || (rc = dalloc(&detmin_e, E, "cudaMalloc(detmin)"))) {
    cudaFree(rho_d);
    cudaFree(detmin_e);
    free_mesh(m);
    return rc;
  }
  cudaMemcpyAsync(m->dD, m->D, sizeof(double) * n * n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(rho_d, m->rho, sizeof(double) * n, cudaMemcpyHostToDevice, st);
  k_coords<<<grid_for(nL, 256), 256, 0, st>>>(p, nL, m->X, m->Y, m->Z);
  k_geom<<<(unsigned)std::min<int64_t>(E, 152 * 16), 256, 0, st>>>(n, E, m->dD, rho_d, m->X, m->Y, m->Z, m->G,
                                                                      m->Gdf, m->B, m->Bdf, detmin_e);
  k_l2g<<<grid_for(nL, 256), 256, 0, st>>>(p, nL, m->l2g);
  k_mask<<<grid_for(m->n_unique, 256), 256, 0, st>>>(p, m->n_unique, m->mask);
  k_l2gm<<<grid_for(nL, 256), 256, 0, st>>>(nL, m->l2g, m->mask, m->l2gm);
  cudaError_t e = cudaGetLastError();
  std::vector<double> dm(E);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dm.data(), detmin_e, sizeof(double) * E, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(rho_d);
  cudaFree(detmin_e);
  if (e != cudaSuccess) {
    rc = sem_cuda_fail(e, "mesh set-up kernels");
    free_mesh(m);
    return rc;
  }
  double dmin = INFINITY;
  for (double v : dm) dmin = std::min(dmin, v);
  m->detJ_min = dmin;
  if (!(dmin > 0.0)) {
    free_mesh(m);
    char buf[128];
    snprintf(buf, sizeof(buf), "sem_mesh_create_box: non-positive Jacobian (min det J = %g)", dmin);
    return sem_fail(SEM_ERR_INVALID_ARG, buf);
  }
  if ((rc = build_gs_tables(m, st)) != SEM_OK || (rc = sem_n1_prepare(m, st)) != SEM_OK) {
    free_mesh(m);
    return rc;
  }
  if (cudaError_t e2 = cudaStreamSynchronize(st)) {
    free_mesh(m);
    return sem_cuda_fail(e2, "sem_mesh_create_box: set-up");
  }
  *out = m;
  return SEM_OK;
}

extern "C" int sem_mesh_destroy(sem_mesh *m) {
  free_mesh(m);
  return SEM_OK;
}

// Host-side audit of a mesh's index tables (the stand-in for a memory
// checker: every index a kernel follows is checked before it is trusted).
extern "C" int sem_mesh_validate(const sem_mesh *m) {
  if (!m) return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_validate: NULL mesh");
  const int64_t nL = m->n_local, nU = m->n_unique;
  std::vector<int32_t> l2g(nL), l2gm(nL), off(nU + 1), perm(nL);
  std::vector<uint8_t> mask(nU);
  std::vector<double> mult(nU);
  SEM_CUDA(cudaMemcpy(l2g.data(), m->l2g, sizeof(int32_t) * nL, cudaMemcpyDeviceToHost));
  SEM_CUDA(cudaMemcpy(l2gm.data(), m->l2gm, sizeof(int32_t) * nL, cudaMemcpyDeviceToHost));
  SEM_CUDA(cudaMemcpy(off.data(), m->gs_off, sizeof(int32_t) * (nU + 1), cudaMemcpyDeviceToHost));
  SEM_CUDA(cudaMemcpy(perm.data(), m->gs_perm, sizeof(int32_t) * nL, cudaMemcpyDeviceToHost));
  SEM_CUDA(cudaMemcpy(mask.data(), m->mask, nU, cudaMemcpyDeviceToHost));
  SEM_CUDA(cudaMemcpy(mult.data(), m->mult, sizeof(double) * nU, cudaMemcpyDeviceToHost));
  char msg[160];
  auto bad = [&](const char *what, int64_t i) {
    snprintf(msg, sizeof(msg), "sem_mesh_validate: %s at index %lld", what, (long long)i);
    return sem_fail(SEM_ERR_INVALID_ARG, msg);
  };
  for (int64_t l = 0; l < nL; ++l) {
    if (l2g[l] < 0 || l2g[l] >= nU) return bad("l2g out of range", l);
    const int32_t want = mask[l2g[l]] ? l2g[l] : -1;
    if (l2gm[l] != want) return bad("l2gm disagrees with l2g and the mask", l);
  }
  if (off[0] != 0 || off[nU] != nL) return bad("CSR offsets do not span the local nodes", 0);
  std::vector<uint8_t> seen(nL, 0);
  for (int64_t g = 0; g < nU; ++g) {
    if (off[g + 1] <= off[g]) return bad("unique node without a copy (CSR offsets not increasing)", g);
    if (mult[g] != (double)(off[g + 1] - off[g])) return bad("multiplicity differs from the copy count", g);
    for (int32_t t = off[g]; t < off[g + 1]; ++t) {
      const int32_t l = perm[t];
      if (l < 0 || l >= nL || seen[l]) return bad("CSR permutation out of range or repeated", t);
      seen[l] = 1;
      if (l2g[l] != g) return bad("CSR segment holds a copy of another node", t);
      if (t > off[g] && perm[t - 1] >= l) return bad("CSR segment not in ascending copy order", t);
    }
  }
  return SEM_OK;
}

extern "C" int sem_mesh_set_deterministic(sem_mesh *m, int on) {
  if (!m) return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_set_deterministic: NULL mesh");
  if (on && !m->det_w) {
    cudaError_t e = cudaMalloc(&m->det_w, sizeof(double) * (size_t)std::max<int64_t>(m->n_local, 1));
    if (e != cudaSuccess) {
      m->det_w = nullptr;
      return sem_cuda_fail(e, "sem_mesh_set_deterministic: cudaMalloc");
    }
  } else if (!on && m->det_w) {
    SEM_CUDA(cudaDeviceSynchronize());  // no launch in flight may still use the scratch
    cudaFree(m->det_w);
    m->det_w = nullptr;
  }
  return SEM_OK;
}

extern "C" int sem_mesh_set_tensor_cores(sem_mesh *m, int on) {
  if (!m) return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_set_tensor_cores: NULL mesh");
  if (on < 0 || on > 2) return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_set_tensor_cores: on must be 0, 1 or 2");
  if (on == 2 && m->n == 8 && !m->Gt) {  // the register-resident route's lane-major copies
    if (int rc = sem_tcr_prepare(m, 0)) return rc;
  }
  m->use_tc = on;
  return SEM_OK;
}

extern "C" int sem_mesh_info_get(const sem_mesh *m, sem_mesh_info *info) {
  if (!m || !info) return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_info_get: NULL argument");
  info->E = m->E;
  info->n_local = m->n_local;
  info->n_unique = m->n_unique;
  info->N = m->N;
  info->detJ_min = m->detJ_min;
  info->X = m->X;
  info->Y = m->Y;
  info->Z = m->Z;
  info->G = m->G;
  info->B = m->B;
  info->l2g = m->l2g;
  info->mask = m->mask;
  info->mult = m->mult;
  return SEM_OK;
}

extern "C" int sem_mesh_copy_maps(const sem_mesh *m, int32_t *l2g_host, uint8_t *mask_host) {
  if (!m) return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_copy_maps: NULL mesh");
  if (l2g_host) SEM_CUDA(cudaMemcpy(l2g_host, m->l2g, sizeof(int32_t) * m->n_local, cudaMemcpyDeviceToHost));
  if (mask_host) SEM_CUDA(cudaMemcpy(mask_host, m->mask, m->n_unique, cudaMemcpyDeviceToHost));
  return SEM_OK;
}

extern "C" int sem_mesh_copy_gs_tables(const sem_mesh *m, int32_t *off_host, int32_t *perm_host) {
  if (!m) return sem_fail(SEM_ERR_INVALID_ARG, "sem_mesh_copy_gs_tables: NULL mesh");
  if (off_host) SEM_CUDA(cudaMemcpy(off_host, m->gs_off, sizeof(int32_t) * (m->n_unique + 1), cudaMemcpyDeviceToHost));
  if (perm_host) SEM_CUDA(cudaMemcpy(perm_host, m->gs_perm, sizeof(int32_t) * m->n_local, cudaMemcpyDeviceToHost));
  return SEM_OK;
}
