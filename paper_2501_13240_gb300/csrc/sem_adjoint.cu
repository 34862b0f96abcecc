// Temperature advection-diffusion with a prescribed velocity history, its
// discrete adjoint, and the bottom-wall Nusselt functional (binary64).
//
// The forward step is the temperature update of the Boussinesq BDF/EXT step
// (Sec. 4.1, Eq. (2); Sec. 2.2: BDF2 for the implicit Helmholtz part, EXT2
// for advection), written with the velocity as input rather than state:
//   T^{n+1} = Tb + H^{-1} M [Q^T B((b1 Q T^n + b2 Q T^{n-1})/dt + a1 N^n + a2 N^{n-1}) - Q^T H_L Q Tb],
//   N^n = -(u^n . grad)(Q T^n) at the local nodes, H = kappa A + (b0/dt) B,
// with BDF1/EXT1 at n = 0 and the Dirichlet lifting Tb = 1 - z/Lz. With the
// velocity frozen, T^K is affine in T^0, so the transposed steps give the
// exact gradient of a linear functional of T^K. Per reverse step n, with
// psi = H^{-1} M g^{n+1} and phi = B Q psi (H, B, Q^T Q symmetric):
//   g^n     += Q^T [(b1/dt) phi + a1 L_n^T phi],
//   g^{n-1} += Q^T [(b2/dt) phi + a2 L_{n-1}^T phi],
//   L^T phi  = -sum_a D_a^T (sum_c (dr_a/dx_c) u_c phi).
// The functional is the mean conductive heat flux through the bottom plate,
//   Nu_b(T) = -(1/A_b) sum_{bottom nodes} rho_i rho_j |x_r x x_s| dT/dz,
// A_b = the same quadrature of 1; it equals 1 for the conduction state.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sem_fields.cuh"
#include "sem_internal.h"

struct sem_tadv {
  const sem_mesh *m = nullptr;
  sem_tadv_params prm;
  int64_t nL = 0, nU = 0;
  double area = 0.0;  // A_b
  double *R = nullptr, *Tb = nullptr, *TbL = nullptr, *wb = nullptr;
  float2 *Rdf = nullptr;  // double-float split of R (SEM_PREC_DF64): the same gradient as the time step
  double *uL[3] = {}, *g[3] = {}, *aL = nullptr, *bL = nullptr, *rhs = nullptr, *x = nullptr;
  double *scal = nullptr;
  double *dinv[2] = {};  // Jacobi inverses of H for the two BDF coefficients b0 (1 and 3/2)
  double key[2] = {-1.0, -1.0};
  void *ws = nullptr;
  size_t ws_bytes = 0;
  std::vector<void *> owned;
};

namespace {

constexpr int kRed = 152 * 2;

struct Coef {
  double b0, b1, b2, a1, a2;
};
Coef coef(int n) {
  if (n == 0) return {1.0, 1.0, 0.0, 1.0, 0.0};  // BDF1/EXT1
  return {1.5, 2.0, -0.5, 2.0, -1.0};            // BDF2/EXT2
}

// rho_i rho_j |x_r x x_s| at the k = 0 nodes of the bottom element layer, 0 elsewhere
__global__ void k_bottom_weights(int n, int64_t E, int64_t plane, const double *__restrict__ D,
                                 const double *__restrict__ rho, const double *__restrict__ X,
                                 const double *__restrict__ Y, const double *__restrict__ Z, double *__restrict__ w) {
  const int n3 = n * n * n;
  const int64_t nL = E * n3;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = l / n3;
    const int q = (int)(l - e * n3);
    const int i = q % n, j = (q / n) % n, k = q / (n * n);
    if (e >= plane || k != 0) {
      w[l] = 0.0;
      continue;
    }
    const int64_t base = e * n3;
    const double *xc[3] = {X + base, Y + base, Z + base};
    double xr[3], xs[3];
    for (int c = 0; c < 3; ++c) {
      double a = 0.0, b = 0.0;
      for (int m = 0; m < n; ++m) {
        a = fma(D[i * n + m], xc[c][m + n * j], a);
        b = fma(D[j * n + m], xc[c][i + n * m], b);
      }
      xr[c] = a;
      xs[c] = b;
    }
    const double cx = xr[1] * xs[2] - xr[2] * xs[1], cy = xr[2] * xs[0] - xr[0] * xs[2],
                 cz = xr[0] * xs[1] - xr[1] * xs[0];
    w[l] = rho[i] * rho[j] * sqrt(cx * cx + cy * cy + cz * cz);
  }
}

// v_a = s w (dr_a/dx_z): the flux functional's weak-form vector
__global__ void k_flux_v(int n, int64_t E, double s, const double *__restrict__ R, const double *__restrict__ w,
                         double *__restrict__ v0, double *__restrict__ v1, double *__restrict__ v2) {
  const int n3 = n * n * n;
  const int64_t nL = E * n3;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = l / n3;
    const int q = (int)(l - e * n3);
    const double *Re = R + 9 * e * n3 + q;
    const double sw = s * w[l];
    v0[l] = sw * Re[0 * n3 + 2 * n3];
    v1[l] = sw * Re[3 * n3 + 2 * n3];
    v2[l] = sw * Re[6 * n3 + 2 * n3];
  }
}

__global__ void k_dot_part(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                           double *__restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[g], y[g], s);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// the forward right-hand side at the local nodes (k.b1, k.b2 divided by dt;
// the same expression as the time step's, so a replayed run repeats it bit for bit)
__global__ void k_rhs_tadv(int64_t nL, Coef k, const double *__restrict__ B, const double *__restrict__ TL,
                           const double *__restrict__ TpL, const double *__restrict__ NT, const double *__restrict__ NTp,
                           const double *__restrict__ HTb, double *__restrict__ out) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x)
    out[l] = B[l] * ((k.b1 * TL[l] + k.b2 * TpL[l]) + (k.a1 * NT[l] + k.a2 * NTp[l])) - HTb[l];
}

// out = c0 phi - c1 s  (s = sum_a D_a^T v_a, so -s = L^T phi)
__global__ void k_adj_combine(int64_t nL, double c0, double c1, const double *phi, const double *s, double *out) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x)
    out[l] = c0 * phi[l] - c1 * s[l];
}

__global__ void k_mul(int64_t n, const double *__restrict__ a, double *__restrict__ x) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    x[g] *= a[g];
}

__global__ void k_mask_copy(int64_t n, const uint8_t *__restrict__ mask, const double *x, double *y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    y[g] = mask[g] ? x[g] : 0.0;
}

void free_tadv(sem_tadv *t) {
  if (!t) return;
  for (void *p : t->owned) cudaFree(p);
  delete t;
}

int solve(sem_tadv *t, double h2, const double *b, double *x, int *iters, cudaStream_t st) {
  sem_solver_opts o;
  o.initial_guess = 0;
  o.tol = t->prm.tol;
  o.maxit = t->prm.maxit;
  o.precision = t->prm.precision;
  o.timeout_s = 0.0;
  o.mask_mode = 0;
  sem_solve_stats stt;
  int slot = (t->key[0] == h2) ? 0 : (t->key[1] == h2) ? 1 : -1;
  if (slot < 0) {  // not cached: fill the slot of this coefficient's step kind
    slot = (h2 == t->key[0] || t->key[0] < 0.0) ? 0 : 1;
    if (int rc = sem_jacobi_inv_mode(t->m, t->prm.kappa, h2, 1, t->dinv[slot], st)) return rc;
    t->key[slot] = h2;
  }
  int rc = sem_pcg_solve_ex(t->m, t->prm.kappa, h2, b, x, &o, t->ws, &stt, (void *)st, 8, t->dinv[slot]);
  if (iters) *iters = stt.iterations;
  return rc;
}

// -(u . grad f) at the local nodes from a local f; velocity already scattered into t->uL
int neg_adv(sem_tadv *t, const double *fL, double *out, cudaStream_t st) {
  const sem_mesh *m = t->m;
  const unsigned gl = grid_for(t->nL, 256);
  if (t->Rdf) {
    if (int rc = sem_launch_grad_df64(m, t->Rdf, fL, t->g[0], t->g[1], t->g[2], st)) return rc;
  } else {
    k_grad<<<gl, 256, 0, st>>>(m->n, m->E, m->dD, t->R, fL, t->g[0], t->g[1], t->g[2]);
  }
  k_neg_adv<<<gl, 256, 0, st>>>(t->nL, t->uL[0], t->uL[1], t->uL[2], t->g[0], t->g[1], t->g[2], nullptr, out);
  SEM_LAUNCH_CHECK("advection");
  return SEM_OK;
}

int scatter_u(sem_tadv *t, const double *const u[3], cudaStream_t st) {
  for (int c = 0; c < 3; ++c)
    if (int rc = sem_launch_scatter(t->m, u[c], t->uL[c], st)) return rc;
  return SEM_OK;
}

// g += Q^T [c0 phi + c1 L^T phi] for the velocity u; phi is local
int adj_acc(sem_tadv *t, const double *const u[3], double c0, double c1, const double *phi, double *g,
            cudaStream_t st) {
  const sem_mesh *m = t->m;
  const unsigned gl = grid_for(t->nL, 256), gu = grid_for(t->nU, 256);
  if (int rc = scatter_u(t, u, st)) return rc;
  k_weak_div_v<<<gl, 256, 0, st>>>(m->n, m->E, t->R, phi, t->uL[0], t->uL[1], t->uL[2], t->g[0], t->g[1], t->g[2]);
  k_dt_sum<<<gl, 256, 0, st>>>(m->n, m->E, m->dD, t->g[0], t->g[1], t->g[2], t->bL);
  k_adj_combine<<<gl, 256, 0, st>>>(t->nL, c0, c1, phi, t->bL, t->bL);
  k_gather_m<<<gu, 256, 0, st>>>(t->nU, m->gs_off, m->gs_perm, nullptr, t->bL, t->rhs);
  k_axpbypcz<<<gu, 256, 0, st>>>(t->nU, 1.0, g, 1.0, t->rhs, 0.0, nullptr, g);
  SEM_LAUNCH_CHECK("adjoint accumulate");
  return SEM_OK;
}

bool bad(const void *p) { return !p || ((uintptr_t)p & 7); }

}  // namespace

extern "C" int sem_tadv_create(const sem_mesh *m, const sem_tadv_params *prm, void *stream, sem_tadv **out) {
  if (!m || !prm || !out) return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_create: NULL argument");
  *out = nullptr;
  if (m->slab) return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_create: needs the whole box, not a partition's slab mesh");
  if (!(prm->kappa > 0) || !(prm->dt > 0) || !(prm->tol > 0) || prm->maxit < 1)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_create: kappa, dt, tol must be > 0 and maxit >= 1");
  if (prm->precision != SEM_PREC_FP64 && prm->precision != SEM_PREC_DF64)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_create: unknown precision");
  int dev = -1;
  SEM_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_create: the mesh's device must be current");
  if (m->periodic[2] || !m->dirichlet[4] || !m->dirichlet[5])
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_create: the mesh needs Dirichlet plates at z = 0 and z = Lz");
  cudaStream_t st = as_stream(stream);
  sem_tadv *t = new sem_tadv();
  t->m = m;
  t->prm = *prm;
  t->nL = m->n_local;
  t->nU = m->n_unique;
  auto alloc = [&](double **p, int64_t count) -> int {
    cudaError_t e = cudaMalloc((void **)p, sizeof(double) * (size_t)std::max<int64_t>(count, 1));
    if (e != cudaSuccess) return sem_cuda_fail(e, "sem_tadv_create: cudaMalloc");
    t->owned.push_back(*p);
    return SEM_OK;
  };
  int rc = SEM_OK;
  double **uvecs[] = {&t->Tb, &t->rhs, &t->x, &t->dinv[0], &t->dinv[1]};
  for (double **p : uvecs)
    if (!rc) rc = alloc(p, t->nU);
  double **evecs[] = {&t->TbL, &t->wb, &t->uL[0], &t->uL[1], &t->uL[2],
                      &t->g[0], &t->g[1],  &t->g[2], &t->aL,    &t->bL};
  for (double **p : evecs)
    if (!rc) rc = alloc(p, t->nL);
  if (!rc) rc = alloc(&t->R, 9 * t->nL);
  if (!rc && prm->precision == SEM_PREC_DF64) {
    cudaError_t e = cudaMalloc((void **)&t->Rdf, sizeof(float2) * 9 * (size_t)std::max<int64_t>(t->nL, 1));
    if (e != cudaSuccess) rc = sem_cuda_fail(e, "sem_tadv_create: cudaMalloc(Rdf)");
    else t->owned.push_back(t->Rdf);
  }
  if (!rc) rc = alloc(&t->scal, kRed + 8 + SEM_MAXNP);
  if (!rc) rc = sem_pcg_workspace_bytes(m, &t->ws_bytes);
  if (!rc) {
    cudaError_t e = cudaMalloc(&t->ws, t->ws_bytes);
    if (e != cudaSuccess) rc = sem_cuda_fail(e, "sem_tadv_create: cudaMalloc(workspace)");
    else t->owned.push_back(t->ws);
  }
  if (rc) {
    free_tadv(t);
    return rc;
  }
  double *drho = t->scal + kRed + 8;
  const unsigned gl = grid_for(t->nL, 256);
  cudaMemcpyAsync(drho, m->rho, sizeof(double) * m->n, cudaMemcpyHostToDevice, st);
  k_inv_jacobian<<<gl, 256, 0, st>>>(m->n, m->E, m->dD, m->X, m->Y, m->Z, t->R);
  if (t->Rdf && (rc = sem_launch_split_df64(t->R, t->Rdf, 9 * t->nL, st))) {
    free_tadv(t);
    return rc;
  }
  k_lifting<<<gl, 256, 0, st>>>(t->nL, m->L[2], m->l2g, m->Z, t->Tb);
  k_bottom_weights<<<gl, 256, 0, st>>>(m->n, m->E, (int64_t)m->nel[0] * m->nel[1], m->dD, drho, m->X, m->Y, m->Z,
                                       t->wb);
  k_sum_part<<<kRed, 256, 0, st>>>(t->nL, t->wb, t->scal);
  k_mean_finish<<<1, 32, 0, st>>>(kRed, 1, t->scal, t->scal + kRed);
  rc = sem_launch_scatter(m, t->Tb, t->TbL, st);
  cudaError_t e = cudaGetLastError();
  if (!rc && e == cudaSuccess) e = cudaMemcpyAsync(&t->area, t->scal + kRed, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (!rc && e != cudaSuccess) rc = sem_cuda_fail(e, "sem_tadv_create: set-up kernels");
  if (rc) {
    free_tadv(t);
    return rc;
  }
  *out = t;
  return SEM_OK;
}

extern "C" int sem_tadv_destroy(sem_tadv *t) {
  free_tadv(t);
  return SEM_OK;
}

extern "C" int sem_tadv_step(sem_tadv *t, int n, const double *const u[3], const double *Tn, const double *Tnm1,
                             const double *NTnm1, double *Tnp1, double *NTn, int *iters, void *stream) {
  SemRange nvtx_range("sem_tadv_step");
  if (!t || !u || n < 0) return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_step: NULL handle/velocity or n < 0");
  if (bad(u[0]) || bad(u[1]) || bad(u[2]) || bad(Tn) || bad(Tnp1) || bad(NTn) ||
      (n > 0 && (bad(Tnm1) || bad(NTnm1))))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_step: NULL or misaligned array");
  cudaStream_t st = as_stream(stream);
  const sem_mesh *m = t->m;
  const unsigned gl = grid_for(t->nL, 256), gu = grid_for(t->nU, 256);
  const Coef k = coef(n);
  int rc;
  if ((rc = scatter_u(t, u, st))) return rc;
  if ((rc = sem_launch_scatter(m, Tn, t->aL, st))) return rc;  // Q T^n
  if ((rc = neg_adv(t, t->aL, NTn, st))) return rc;             // N^n
  const double *TpL = t->aL, *NTp = NTn;                         // n = 0: the history is the current level
  if (n > 0) {
    if ((rc = sem_launch_scatter(m, Tnm1, t->bL, st))) return rc;
    TpL = t->bL;
    NTp = NTnm1;
  }
  // H_L Tb with h2 = b0/dt
  if ((rc = sem_launch_ax_local(m, t->prm.kappa, k.b0 / t->prm.dt, t->TbL, t->g[0], t->prm.precision, st)))
    return rc;
  Coef kd = k;
  kd.b1 = k.b1 / t->prm.dt;
  kd.b2 = k.b2 / t->prm.dt;
  k_rhs_tadv<<<gl, 256, 0, st>>>(t->nL, kd, m->B, t->aL, TpL, NTn, NTp, t->g[0], t->g[2]);
  k_gather_m<<<gu, 256, 0, st>>>(t->nU, m->gs_off, m->gs_perm, m->mask, t->g[2], t->rhs);
  SEM_LAUNCH_CHECK("tadv right-hand side");
  int it = 0;
  rc = solve(t, k.b0 / t->prm.dt, t->rhs, t->x, &it, st);
  if (iters) *iters = it;
  if (rc && rc != SEM_ERR_NOT_CONVERGED) return rc;
  k_axpbypcz<<<gu, 256, 0, st>>>(t->nU, 1.0, t->Tb, 1.0, t->x, 0.0, nullptr, Tnp1);
  SEM_LAUNCH_CHECK("tadv update");
  SEM_CUDA(cudaStreamSynchronize(st));
  return rc;
}

extern "C" int sem_tadv_adjoint_step(sem_tadv *t, int n, const double *const u_n[3], const double *const u_nm1[3],
                                     const double *g_np1, double *g_n, double *g_nm1, int *iters, void *stream) {
  SemRange nvtx_range("sem_tadv_adjoint_step");
  if (!t || !u_n || n < 0) return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_adjoint_step: NULL handle/velocity or n < 0");
  if (bad(u_n[0]) || bad(u_n[1]) || bad(u_n[2]) || bad(g_np1) || bad(g_n) ||
      (n > 0 && (!u_nm1 || bad(u_nm1[0]) || bad(u_nm1[1]) || bad(u_nm1[2]) || bad(g_nm1))))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_adjoint_step: NULL or misaligned array");
  cudaStream_t st = as_stream(stream);
  const sem_mesh *m = t->m;
  const unsigned gu = grid_for(t->nU, 256);
  const Coef k = coef(n);
  const double dt = t->prm.dt;
  int rc;
  // psi = H^{-1} M g^{n+1}, phi = B Q psi
  k_mask_copy<<<gu, 256, 0, st>>>(t->nU, m->mask, g_np1, t->rhs);
  SEM_LAUNCH_CHECK("k_mask_copy");
  int it = 0;
  rc = solve(t, k.b0 / dt, t->rhs, t->x, &it, st);
  if (iters) *iters = it;
  if (rc && rc != SEM_ERR_NOT_CONVERGED) return rc;
  const int solve_rc = rc;
  if ((rc = sem_launch_scatter(m, t->x, t->aL, st))) return rc;
  k_mul<<<grid_for(t->nL, 256), 256, 0, st>>>(t->nL, m->B, t->aL);
  SEM_LAUNCH_CHECK("k_mul");
  if ((rc = adj_acc(t, u_n, k.b1 / dt, k.a1, t->aL, g_n, st))) return rc;
  if (n > 0 && (rc = adj_acc(t, u_nm1, k.b2 / dt, k.a2, t->aL, g_nm1, st))) return rc;
  if (n == 0) {  // g^0 is the gradient with respect to the free values of T^0
    k_mask_copy<<<gu, 256, 0, st>>>(t->nU, m->mask, g_n, g_n);
    SEM_LAUNCH_CHECK("k_mask_copy");
  }
  SEM_CUDA(cudaStreamSynchronize(st));
  return solve_rc;
}

extern "C" int sem_tadv_nusselt(sem_tadv *t, const double *T, double *nu, void *stream) {
  if (!t || bad(T) || !nu) return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_nusselt: NULL or misaligned argument");
  cudaStream_t st = as_stream(stream);
  const sem_mesh *m = t->m;
  const unsigned gl = grid_for(t->nL, 256);
  int rc;
  if ((rc = sem_launch_scatter(m, T, t->aL, st))) return rc;
  k_grad<<<gl, 256, 0, st>>>(m->n, m->E, m->dD, t->R, t->aL, t->g[0], t->g[1], t->g[2]);
  k_dot_part<<<kRed, 256, 0, st>>>(t->nL, t->wb, t->g[2], t->scal);
  k_mean_finish<<<1, 32, 0, st>>>(kRed, 1, t->scal, t->scal + kRed);
  SEM_LAUNCH_CHECK("nusselt");
  double s = 0.0;
  SEM_CUDA(cudaMemcpyAsync(&s, t->scal + kRed, sizeof(double), cudaMemcpyDeviceToHost, st));
  SEM_CUDA(cudaStreamSynchronize(st));
  *nu = -s / t->area;
  return SEM_OK;
}

extern "C" int sem_tadv_nusselt_grad(sem_tadv *t, double scale, double *c, void *stream) {
  if (!t || bad(c)) return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_nusselt_grad: NULL or misaligned argument");
  cudaStream_t st = as_stream(stream);
  const sem_mesh *m = t->m;
  const unsigned gl = grid_for(t->nL, 256);
  k_flux_v<<<gl, 256, 0, st>>>(m->n, m->E, -scale / t->area, t->R, t->wb, t->g[0], t->g[1], t->g[2]);
  k_dt_sum<<<gl, 256, 0, st>>>(m->n, m->E, m->dD, t->g[0], t->g[1], t->g[2], t->aL);
  k_gather_m<<<grid_for(t->nU, 256), 256, 0, st>>>(t->nU, m->gs_off, m->gs_perm, nullptr, t->aL, c);
  SEM_LAUNCH_CHECK("nusselt gradient");
  SEM_CUDA(cudaStreamSynchronize(st));
  return SEM_OK;
}

extern "C" int sem_tadv_info(const sem_tadv *t, double *area, const double **Tb) {
  if (!t) return sem_fail(SEM_ERR_INVALID_ARG, "sem_tadv_info: NULL handle");
  if (area) *area = t->area;
  if (Tb) *Tb = t->Tb;
  return SEM_OK;
}
