// One rank's share of an element-slab partition on its GPU, and the
// assembled operator and Jacobi-PCG over the partition (Sec. 2.2: one rank
// per GPU; shared surface values are summed across ranks, and the exchange
// is overlapped with the interior work: surface elements first, start the
// exchange, interior elements, finish the surface nodes).
//
// The rank holds a slab mesh: its element planes of the box with its own
// unique numbering (lattice planes p0 N .. p1 N, no periodic wrap in z), so
// its vectors have only its own nodes. The nodes it shares with other ranks
// (the interface, sem_partition_interface) are its first and/or last
// lattice plane; only the elements of its first and last element plane (the
// surface elements, sem_partition_surface) touch them.
//
// Operator, per application:
//   stream A: w = 0; surface elements; gather the interface values; D2H
//   stream B: (after w = 0) interior elements        -- runs during the exchange
//   host:     the caller's exchange callback sums the interface values over
//             the ranks (in place, in ascending unique-id order of the box)
//   stream A: H2D; the full sums written to the interface nodes; join B
// Interior elements touch no interface node, so the two streams never add
// into the same node, and the sums written last are complete.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "sem_internal.h"

struct sem_part {
  sem_mesh *m = nullptr;  // the slab mesh (owned)
  int nranks = 1, rank = 0;
  int64_t e_begin = 0, e_end = 0;  // the slab's elements in the box's numbering
  int64_t n_surf = 0, n_int = 0, n_if = 0;
  int32_t *d_surf = nullptr, *d_int = nullptr;  // local element ids
  int32_t *d_if = nullptr;                      // local unique ids of the interface nodes (box id order)
  double *d_wdot = nullptr;                     // inner-product weight of each local node (1 / ranks holding it)
  double *d_buf = nullptr;                      // interface values (device)
  double *h_buf = nullptr;                      // interface values (pinned host)
  double *d_part = nullptr;                     // reduction partials
  double *d_vec = nullptr;                      // r, p, w, z, dinv of the partitioned solve
  double *h_part = nullptr;                     // pinned copy of the reduced scalars
  cudaStream_t s2 = nullptr;                    // the interior elements' stream
  cudaEvent_t ev_clear = nullptr, ev_int = nullptr;
};

namespace {

constexpr int kRedBlocks = 152 * 2, kRedThreads = 256;

__global__ void k_take(int64_t n, const int32_t *__restrict__ idx, const double *__restrict__ v, double *__restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v[idx[i]];
}

__global__ void k_put(int64_t n, const int32_t *__restrict__ idx, const double *__restrict__ in, double *__restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[idx[i]] = in[i];
}

__global__ void k_fill_d(int64_t n, double a, double *__restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) v[i] = a;
}

__global__ void k_put_scalar(int64_t n, const int32_t *__restrict__ idx, const double *__restrict__ vals,
                             double *__restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[idx[i]] = vals[i];
}

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int t = 0; t < (int)(blockDim.x >> 5); ++t) s += red[t];  // every thread, same order
  return s;
}

template <int K>
struct VecPairs {
  const double *a[K], *b[K];
};

// k partial sums of weighted products: slot q of block b = sum wdot a_q b_q
template <int K>
__global__ void __launch_bounds__(kRedThreads)
    k_wdots(int64_t n, const double *__restrict__ wdot, VecPairs<K> v, double *__restrict__ part) {
  const double *const *a = v.a, *const *b = v.b;
  __shared__ double red[32];
  double s[K];
#pragma unroll
  for (int q = 0; q < K; ++q) s[q] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = wdot[i];
#pragma unroll
    for (int q = 0; q < K; ++q) s[q] = fma(wi * a[q][i], b[q][i], s[q]);
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const double t = block_sum(s[q], red);
    if (threadIdx.x == 0) part[q * gridDim.x + blockIdx.x] = t;
  }
}

// out[q] = sum over blocks of part[q][.] (one CTA, fixed order)
__global__ void __launch_bounds__(kRedThreads) k_finish(int k, int nb, const double *__restrict__ part, double *out) {
  __shared__ double red[32];
  for (int q = 0; q < k; ++q) {
    double s = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) s += part[q * nb + t];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[q] = s;
  }
}

// x += alpha p; r -= alpha w; (z = dinv r recomputed where needed)
__global__ void k_upd1(int64_t n, double alpha, const double *__restrict__ p, const double *__restrict__ w,
                       double *__restrict__ x, double *__restrict__ r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, w[i], r[i]);
  }
}

__global__ void k_zr(int64_t n, const double *__restrict__ dinv, const double *__restrict__ r, double *__restrict__ z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = dinv[i] * r[i];
}

__global__ void k_upd2(int64_t n, double beta, const double *__restrict__ z, double *__restrict__ p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

// assembled diagonal over the slab's copies (not yet summed across ranks)
__global__ void k_diag_slab(int n, int64_t nU, const int32_t *__restrict__ off, const int32_t *__restrict__ perm,
                            const double *__restrict__ Dg, const double *__restrict__ G, const double *__restrict__ B,
                            double h1, double h2, double *__restrict__ d) {
  const int n3 = n * n * n;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nU; g += (int64_t)gridDim.x * blockDim.x) {
    double tot = 0.0;
    for (int32_t t = off[g]; t < off[g + 1]; ++t) {
      const int64_t l = perm[t];
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
      tot += h1 * s + h2 * B[l];
    }
    d[g] = tot;
  }
}

__global__ void k_invert_masked(int64_t n, const uint8_t *__restrict__ mask, double *__restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = mask[i] ? 1.0 / d[i] : 0.0;
}

void free_part(sem_part *p) {
  if (!p) return;
  if (p->m) sem_mesh_destroy(p->m);
  void *dev[] = {p->d_surf, p->d_int, p->d_if, p->d_wdot, p->d_buf, p->d_part, p->d_vec};
  for (void *q : dev)
    if (q) cudaFree(q);
  if (p->h_buf) cudaFreeHost(p->h_buf);
  if (p->h_part) cudaFreeHost(p->h_part);
  if (p->s2) cudaStreamDestroy(p->s2);
  if (p->ev_clear) cudaEventDestroy(p->ev_clear);
  if (p->ev_int) cudaEventDestroy(p->ev_int);
  delete p;
}

int exchange_fail(int rc) {
  return sem_fail(SEM_ERR_IO, "partitioned operator: the exchange callback returned " + std::to_string(rc));
}

// w = M Q^T A Q M u over the rank's nodes with the overlapped exchange
int part_ax(sem_part *P, double h1, double h2, const double *u, double *w, int precision, sem_exchange_fn ex,
            void *user, cudaStream_t st) {
  const sem_mesh *m = P->m;
  SEM_CUDA(cudaMemsetAsync(w, 0, sizeof(double) * m->n_unique, st));
  SEM_CUDA(cudaEventRecord(P->ev_clear, st));
  int rc;
  if ((rc = sem_launch_ax_assembled_list(m, h1, h2, u, w, precision, st, P->d_surf, P->n_surf))) return rc;
  if (P->n_if > 0) {
    k_take<<<grid_for(P->n_if, 256), 256, 0, st>>>(P->n_if, P->d_if, w, P->d_buf);
    SEM_LAUNCH_CHECK("interface gather");
    SEM_CUDA(cudaMemcpyAsync(P->h_buf, P->d_buf, sizeof(double) * P->n_if, cudaMemcpyDeviceToHost, st));
  }
  SEM_CUDA(cudaStreamWaitEvent(P->s2, P->ev_clear, 0));
  if ((rc = sem_launch_ax_assembled_list(m, h1, h2, u, w, precision, P->s2, P->d_int, P->n_int))) return rc;
  SEM_CUDA(cudaEventRecord(P->ev_int, P->s2));
  if (P->n_if > 0) {
    SEM_CUDA(cudaStreamSynchronize(st));  // the partial sums have arrived (the interior runs on)
    if (int e = ex(P->h_buf, P->n_if, user)) {
      cudaStreamSynchronize(P->s2);
      return exchange_fail(e);
    }
    SEM_CUDA(cudaMemcpyAsync(P->d_buf, P->h_buf, sizeof(double) * P->n_if, cudaMemcpyHostToDevice, st));
    k_put<<<grid_for(P->n_if, 256), 256, 0, st>>>(P->n_if, P->d_if, P->d_buf, w);
    SEM_LAUNCH_CHECK("interface scatter");
  }
  SEM_CUDA(cudaStreamWaitEvent(st, P->ev_int, 0));
  return SEM_OK;
}

// k weighted inner products over the rank's nodes, summed over the ranks
template <int K>
int wdots(sem_part *P, const double *const (&a)[K], const double *const (&b)[K], double (&out)[K], sem_allreduce_fn ar,
          void *user, cudaStream_t st) {
  const int64_t n = P->m->n_unique;
  VecPairs<K> v;
  for (int q = 0; q < K; ++q) {
    v.a[q] = a[q];
    v.b[q] = b[q];
  }
  k_wdots<K><<<kRedBlocks, kRedThreads, 0, st>>>(n, P->d_wdot, v, P->d_part);
  k_finish<<<1, kRedThreads, 0, st>>>(K, kRedBlocks, P->d_part, P->d_part + 3 * kRedBlocks);
  SEM_LAUNCH_CHECK("weighted inner products");
  SEM_CUDA(cudaMemcpyAsync(P->h_part, P->d_part + 3 * kRedBlocks, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
  SEM_CUDA(cudaStreamSynchronize(st));
  if (P->nranks > 1)
    if (int e = ar(P->h_part, K, user)) return sem_fail(SEM_ERR_IO, "partitioned solve: the all-reduce callback failed");
  for (int q = 0; q < K; ++q) out[q] = P->h_part[q];
  return SEM_OK;
}

int check_part(const sem_part *p, const char *fn) {
  if (!p) return sem_fail(SEM_ERR_INVALID_ARG, std::string(fn) + ": NULL partition");
  return SEM_OK;
}

}  // namespace

extern "C" int sem_part_create(const sem_box_desc *desc, int nranks, int rank, void *stream, sem_part **out) {
  SemRange nvtx_range("sem_part_create");
  if (!out) return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_create: NULL output");
  *out = nullptr;
  int64_t e0, e1, nif;
  if (int rc = sem_partition_info(desc, nranks, rank, &e0, &e1, &nif)) return rc;
  const int64_t plane = (int64_t)desc->nelx * desc->nely;
  sem_part *P = new sem_part();
  P->nranks = nranks;
  P->rank = rank;
  P->e_begin = e0;
  P->e_end = e1;
  cudaStream_t st = as_stream(stream);
  int rc;
  if ((rc = sem_mesh_create_slab(desc, (int)(e0 / plane), (int)(e1 / plane), stream, &P->m))) {
    free_part(P);
    return rc;
  }
  const sem_mesh *m = P->m;
  // the plan: surface elements, interface nodes (box ids, ascending) and
  // how many ranks hold each
  std::vector<int64_t> surf(e1 - e0), gids(nif);
  std::vector<int32_t> nshare(nif);
  int64_t nsurf = 0;
  if ((rc = sem_partition_surface(desc, nranks, rank, surf.data(), &nsurf)) ||
      (nif > 0 && (rc = sem_partition_interface(desc, nranks, rank, gids.data(), nshare.data())))) {
    free_part(P);
    return rc;
  }
  std::vector<uint8_t> is_surf(e1 - e0, 0);
  std::vector<int32_t> hs, hi;
  for (int64_t i = 0; i < nsurf; ++i) is_surf[surf[i] - e0] = 1;
  for (int64_t e = 0; e < e1 - e0; ++e) (is_surf[e] ? hs : hi).push_back((int32_t)e);
  // box id -> the slab's id: same I, J; plane K (box, wrapped) -> K - p0 N,
  // where the wrapped plane 0 of a periodic z is the slab's top plane
  const int64_t nx = (int64_t)desc->nelx * desc->N + (desc->periodic[0] ? 0 : 1);
  const int64_t ny = (int64_t)desc->nely * desc->N + (desc->periodic[1] ? 0 : 1);
  const int64_t k0 = (e0 / plane) * desc->N, k1 = (e1 / plane) * desc->N;
  std::vector<int32_t> lif(nif);
  std::vector<double> wif(nif);
  for (int64_t i = 0; i < nif; ++i) {
    const int64_t g = gids[i];
    const int64_t I = g % nx, J = (g / nx) % ny;
    int64_t K = g / (nx * ny);
    if (K < k0 || K > k1) K += (int64_t)desc->nelz * desc->N;  // the periodic wrap
    if (K < k0 || K > k1) {
      free_part(P);
      return sem_fail(SEM_ERR_CUDA, "sem_part_create: interface node outside the slab (plan inconsistent)");
    }
    lif[i] = (int32_t)(I + nx * (J + ny * (K - k0)));
    wif[i] = 1.0 / nshare[i];
  }
  P->n_surf = (int64_t)hs.size();
  P->n_int = (int64_t)hi.size();
  P->n_if = nif;
  auto dal = [](void **p, size_t b) { return cudaMalloc(p, b ? b : 8); };
  cudaError_t e = dal((void **)&P->d_surf, sizeof(int32_t) * hs.size());
  if (e == cudaSuccess) e = dal((void **)&P->d_int, sizeof(int32_t) * hi.size());
  if (e == cudaSuccess) e = dal((void **)&P->d_if, sizeof(int32_t) * nif);
  if (e == cudaSuccess) e = dal((void **)&P->d_wdot, sizeof(double) * m->n_unique);
  if (e == cudaSuccess) e = dal((void **)&P->d_buf, sizeof(double) * nif);
  if (e == cudaSuccess) e = dal((void **)&P->d_part, sizeof(double) * (4 * kRedBlocks + 16));
  if (e == cudaSuccess) e = dal((void **)&P->d_vec, sizeof(double) * 5 * (size_t)m->n_unique);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&P->h_buf, sizeof(double) * std::max<int64_t>(nif, 1));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&P->h_part, sizeof(double) * 8);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->s2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_clear, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_int, cudaEventDisableTiming);
  if (e == cudaSuccess && !hs.empty())
    e = cudaMemcpyAsync(P->d_surf, hs.data(), sizeof(int32_t) * hs.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !hi.empty())
    e = cudaMemcpyAsync(P->d_int, hi.data(), sizeof(int32_t) * hi.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nif > 0)
    e = cudaMemcpyAsync(P->d_if, lif.data(), sizeof(int32_t) * nif, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nif > 0)
    e = cudaMemcpyAsync(P->d_buf, wif.data(), sizeof(double) * nif, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_fill_d<<<grid_for(m->n_unique, 256), 256, 0, st>>>(m->n_unique, 1.0, P->d_wdot);
    if (nif > 0) k_put_scalar<<<grid_for(nif, 256), 256, 0, st>>>(nif, P->d_if, P->d_buf, P->d_wdot);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_part(P);
    return sem_cuda_fail(e, "sem_part_create");
  }
  *out = P;
  return SEM_OK;
}

extern "C" int sem_part_destroy(sem_part *p) {
  if (p) {
    cudaStreamSynchronize(p->s2);
    free_part(p);
  }
  return SEM_OK;
}

extern "C" int sem_part_info(const sem_part *p, sem_part_info_t *info) {
  if (int rc = check_part(p, "sem_part_info")) return rc;
  if (!info) return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_info: NULL output");
  info->mesh = p->m;
  info->e_begin = p->e_begin;
  info->e_end = p->e_end;
  info->n_surface = p->n_surf;
  info->n_interior = p->n_int;
  info->n_interface = p->n_if;
  info->n_unique = p->m->n_unique;
  return SEM_OK;
}

extern "C" int sem_part_global_ids(const sem_part *p, int64_t *gids_host) {
  if (int rc = check_part(p, "sem_part_global_ids")) return rc;
  if (!gids_host) return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_global_ids: NULL output");
  const sem_box_desc &d = p->m->desc;
  const int64_t nx = (int64_t)d.nelx * d.N + (d.periodic[0] ? 0 : 1);
  const int64_t ny = (int64_t)d.nely * d.N + (d.periodic[1] ? 0 : 1);
  const int64_t Kmax = (int64_t)d.nelz * d.N;
  const int64_t k0 = (int64_t)p->m->slab_p0 * d.N;
  for (int64_t l = 0; l < p->m->n_unique; ++l) {
    const int64_t I = l % nx, J = (l / nx) % ny;
    int64_t K = l / (nx * ny) + k0;
    if (d.periodic[2] && K == Kmax) K = 0;
    gids_host[l] = I + nx * (J + ny * K);
  }
  return SEM_OK;
}

extern "C" int sem_ax_assembled_elems(const sem_mesh *m, double h1, double h2, const double *u_g, double *w_g,
                                      const int32_t *elems, int64_t n_elems, int precision, void *stream) {
  SemRange nvtx_range("sem_ax_assembled_elems");
  if (!m) return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_elems: NULL mesh");
  if (!u_g || !w_g || ((uintptr_t)u_g & 7) || ((uintptr_t)w_g & 7))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_elems: NULL or misaligned vector");
  if (u_g == w_g) return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_elems: u_g and w_g must not overlap");
  if (n_elems < 0 || (n_elems > 0 && !elems) || n_elems > m->E)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_elems: bad element list");
  if (precision != SEM_PREC_FP64 && precision != SEM_PREC_DF64)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_elems: unknown precision");
  return sem_launch_ax_assembled_list(m, h1, h2, u_g, w_g, precision, as_stream(stream), elems, n_elems);
}

extern "C" int sem_part_ax(sem_part *p, double h1, double h2, const double *u, double *w, int precision,
                           sem_exchange_fn ex, void *user, void *stream) {
  SemRange nvtx_range("sem_part_ax");
  if (int rc = check_part(p, "sem_part_ax")) return rc;
  if (!u || !w || ((uintptr_t)u & 7) || ((uintptr_t)w & 7) || u == w)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_ax: NULL, misaligned or overlapping vectors");
  if (p->n_if > 0 && !ex) return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_ax: NULL exchange callback");
  if (precision != SEM_PREC_FP64 && precision != SEM_PREC_DF64)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_ax: unknown precision");
  return part_ax(p, h1, h2, u, w, precision, ex, user, as_stream(stream));
}

extern "C" int sem_part_pcg_solve(sem_part *p, double h1, double h2, const double *b, double *x,
                                  const sem_solver_opts *opts, sem_solve_stats *stats, sem_exchange_fn ex,
                                  sem_allreduce_fn ar, void *user, void *stream) {
  SemRange nvtx_range("sem_part_pcg_solve");
  if (int rc = check_part(p, "sem_part_pcg_solve")) return rc;
  if (!b || !x || ((uintptr_t)b & 7) || ((uintptr_t)x & 7) || b == x)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_pcg_solve: NULL, misaligned or overlapping vectors");
  if (!opts || !stats) return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_pcg_solve: NULL opts or stats");
  if ((p->n_if > 0 && !ex) || (p->nranks > 1 && !ar))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_pcg_solve: NULL exchange or all-reduce callback");
  if (!(opts->tol >= 0.0) || opts->maxit < 1 || opts->mask_mode != 0)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_pcg_solve: bad tol, maxit or mask_mode (Dirichlet only)");
  if (opts->initial_guess != 0)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_pcg_solve: starts from x = 0 (initial_guess must be 0)");
  if (opts->precision != SEM_PREC_FP64 && opts->precision != SEM_PREC_DF64)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_pcg_solve: unknown precision");
  if (!(h1 >= 0.0) || !(h2 >= 0.0) || (h1 == 0.0 && h2 == 0.0))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_part_pcg_solve: need h1 >= 0, h2 >= 0, not both zero");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = as_stream(stream);
  const sem_mesh *m = p->m;
  const int64_t n = m->n_unique;
  stats->iterations = 0;
  stats->rel_residual = 0.0;
  stats->status = SEM_OK;
  double *r = p->d_vec, *pp = nullptr, *w = nullptr, *z = nullptr, *dinv = nullptr;
  cudaError_t e = cudaSuccess;
  pp = r + n;
  w = pp + n;
  z = w + n;
  dinv = z + n;
  int rc = SEM_OK, it = 0;
  double rr = 0.0, bnorm = 0.0;
  const unsigned gv = grid_for(n, 256);
  do {
    // Jacobi diagonal: the slab's sums, completed across the ranks, inverted on free nodes
    k_diag_slab<<<gv, 256, 0, st>>>(m->n, n, m->gs_off, m->gs_perm, m->dD, m->G, m->B, h1, h2, dinv);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      rc = sem_cuda_fail(e, "partitioned diagonal");
      break;
    }
    if (p->n_if > 0) {
      k_take<<<grid_for(p->n_if, 256), 256, 0, st>>>(p->n_if, p->d_if, dinv, p->d_buf);
      if ((e = cudaMemcpyAsync(p->h_buf, p->d_buf, sizeof(double) * p->n_if, cudaMemcpyDeviceToHost, st)) ||
          (e = cudaStreamSynchronize(st))) {
        rc = sem_cuda_fail(e, "partitioned diagonal");
        break;
      }
      if (int x_ = ex(p->h_buf, p->n_if, user)) {
        rc = exchange_fail(x_);
        break;
      }
      cudaMemcpyAsync(p->d_buf, p->h_buf, sizeof(double) * p->n_if, cudaMemcpyHostToDevice, st);
      k_put<<<grid_for(p->n_if, 256), 256, 0, st>>>(p->n_if, p->d_if, p->d_buf, dinv);
    }
    k_invert_masked<<<gv, 256, 0, st>>>(n, m->mask, dinv);
    // x = 0, r = b, z = dinv r, p = z
    cudaMemsetAsync(x, 0, sizeof(double) * n, st);
    cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    k_zr<<<gv, 256, 0, st>>>(n, dinv, r, z);
    cudaMemcpyAsync(pp, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      rc = sem_cuda_fail(e, "partitioned solve set-up");
      break;
    }
    double s2[2];
    if ((rc = wdots<2>(p, {b, r}, {b, z}, s2, ar, user, st))) break;
    bnorm = sqrt(s2[0]);
    double rho = s2[1];
    rr = s2[0];
    if (!(bnorm > 0.0)) break;  // b = 0: x = 0
    const double thresh = opts->tol * bnorm;
    rc = SEM_ERR_NOT_CONVERGED;
    for (it = 1; it <= opts->maxit; ++it) {
      int r2;
      if ((r2 = part_ax(p, h1, h2, pp, w, opts->precision, ex, user, st))) {
        rc = r2;
        break;
      }
      double s1[1];
      if ((r2 = wdots<1>(p, {pp}, {w}, s1, ar, user, st))) {
        rc = r2;
        break;
      }
      const double pw = s1[0];
      if (!(pw > 0.0) || !std::isfinite(pw)) {
        rc = SEM_ERR_BREAKDOWN;
        break;
      }
      const double alpha = rho / pw;
      k_upd1<<<gv, 256, 0, st>>>(n, alpha, pp, w, x, r);
      k_zr<<<gv, 256, 0, st>>>(n, dinv, r, z);
      if ((r2 = wdots<2>(p, {r, r}, {z, r}, s2, ar, user, st))) {
        rc = r2;
        break;
      }
      rr = s2[1];
      if (std::isfinite(rr) && sqrt(rr) <= thresh) {
        rc = SEM_OK;
        break;
      }
      if (!std::isfinite(rr) || !std::isfinite(s2[0])) {
        rc = SEM_ERR_BREAKDOWN;
        break;
      }
      const double beta = s2[0] / rho;
      rho = s2[0];
      k_upd2<<<gv, 256, 0, st>>>(n, beta, z, pp);
      if (opts->timeout_s > 0.0 &&
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > opts->timeout_s) {
        rc = SEM_ERR_TIMEOUT;
        break;
      }
    }
    if (it > opts->maxit) it = opts->maxit;
  } while (0);
  cudaStreamSynchronize(st);
  stats->iterations = it;
  stats->rel_residual = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
  stats->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  stats->status = rc;
  if (rc == SEM_ERR_NOT_CONVERGED) sem_fail(rc, "sem_part_pcg_solve: maxit reached");
  if (rc == SEM_ERR_BREAKDOWN) sem_fail(rc, "sem_part_pcg_solve: breakdown (p.Ap <= 0 or non-finite)");
  if (rc == SEM_ERR_TIMEOUT) sem_fail(rc, "sem_part_pcg_solve: timeout");
  return rc;
}
