// Direct stiffness summation (gather-scatter): Q^T sums the local copies of
// each unique node, Q copies unique values back. The paper's ranks exchange
// and sum shared surface values (Sec. 2.2); on one GPU the same summation is
// a deterministic CSR gather over the unique nodes.
#include "sem_internal.h"

namespace {

__global__ void k_gs_csr(int64_t nU, const int32_t *__restrict__ off, const int32_t *__restrict__ perm,
                         const uint8_t *__restrict__ mask, int apply_mask, double *__restrict__ v) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nU; g += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = off[g], b = off[g + 1];
    double s = 0.0;
    for (int32_t t = a; t < b; ++t) s += v[perm[t]];
    if (apply_mask && !mask[g]) s = 0.0;
    for (int32_t t = a; t < b; ++t) v[perm[t]] = s;
  }
}

__global__ void k_gather(int64_t nU, const int32_t *__restrict__ off, const int32_t *__restrict__ perm,
                         const double *__restrict__ vL, double *__restrict__ vg) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nU; g += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = off[g], b = off[g + 1];
    double s = 0.0;
    for (int32_t t = a; t < b; ++t) s += vL[perm[t]];
    vg[g] = s;
  }
}

__global__ void k_scatter(int64_t nL, const int32_t *__restrict__ l2g, const double *__restrict__ vg,
                          double *__restrict__ vL) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x)
    vL[l] = vg[l2g[l]];
}

__global__ void k_weak_rhs(int64_t nU, const int32_t *__restrict__ off, const int32_t *__restrict__ perm,
                           const uint8_t *__restrict__ mask, const double *__restrict__ B,
                           const double *__restrict__ f, double *__restrict__ b) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nU; g += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int32_t t = off[g]; t < off[g + 1]; ++t) {
      const int32_t l = perm[t];
      s = fma(B[l], f[l], s);
    }
    b[g] = mask[g] ? s : 0.0;
  }
}

}  // namespace

extern "C" int sem_weak_rhs(const sem_mesh *m, const double *f_L, double *b_g, void *stream) {
  if (!m || !f_L || !b_g) return sem_fail(SEM_ERR_INVALID_ARG, "sem_weak_rhs: NULL argument");
  k_weak_rhs<<<grid_for(m->n_unique, 256), 256, 0, as_stream(stream)>>>(m->n_unique, m->gs_off, m->gs_perm, m->mask,
                                                                        m->B, f_L, b_g);
  SEM_LAUNCH_CHECK("k_weak_rhs");
  return SEM_OK;
}

int sem_launch_gs(const sem_mesh *m, double *v, int apply_mask, cudaStream_t st) {
  k_gs_csr<<<grid_for(m->n_unique, 256), 256, 0, st>>>(m->n_unique, m->gs_off, m->gs_perm, m->mask, apply_mask, v);
  SEM_LAUNCH_CHECK("k_gs_csr");
  return SEM_OK;
}

namespace {
template <typename T>
__global__ void k_gather_add(int64_t nU, const int32_t *__restrict__ off, const int32_t *__restrict__ perm,
                             const T *__restrict__ wL, T *__restrict__ w) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nU; g += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = off[g], b = off[g + 1];
    T s = T(0);
    for (int32_t t = a; t < b; ++t) s += wL[perm[t]];
    w[g] += s;
  }
}
}  // namespace

int sem_launch_gather_add(const sem_mesh *m, const double *wL, double *w, cudaStream_t st) {
  k_gather_add<double><<<grid_for(m->n_unique, 256), 256, 0, st>>>(m->n_unique, m->gs_off, m->gs_perm, wL, w);
  SEM_LAUNCH_CHECK("k_gather_add");
  return SEM_OK;
}

int sem_launch_gather_add_f(const sem_mesh *m, const float *wL, float *w, cudaStream_t st) {
  k_gather_add<float><<<grid_for(m->n_unique, 256), 256, 0, st>>>(m->n_unique, m->gs_off, m->gs_perm, wL, w);
  SEM_LAUNCH_CHECK("k_gather_add");
  return SEM_OK;
}

int sem_launch_gather(const sem_mesh *m, const double *vL, double *vg, cudaStream_t st) {
  k_gather<<<grid_for(m->n_unique, 256), 256, 0, st>>>(m->n_unique, m->gs_off, m->gs_perm, vL, vg);
  SEM_LAUNCH_CHECK("k_gather");
  return SEM_OK;
}

int sem_launch_scatter(const sem_mesh *m, const double *vg, double *vL, cudaStream_t st) {
  k_scatter<<<grid_for(m->n_local, 256), 256, 0, st>>>(m->n_local, m->l2g, vg, vL);
  SEM_LAUNCH_CHECK("k_scatter");
  return SEM_OK;
}
