// One BDF2/EXT2 time step of the Boussinesq equations (Sec. 4.1, Eqs. (1)-(3))
// for Rayleigh-Benard convection: periodic x, y; isothermal no-slip plates
// (Sec. 4.4). The paper gives no splitting scheme (it names NekRS and its
// pressure Poisson solve, Sec. 2.2); this follows the high-order splitting of
// the spectral-element textbook it cites, in weak form, step n -> n+1:
//   explicit terms at t^n collocated at the GLL nodes: N_T = -u.grad T,
//     N_u = -(u.grad)u + T z, wall term W = nu sum_walls (phi n.curl curl u)
//     with element-local derivatives; EXT2 X* = 2 X^n - X^{n-1};
//   T:  (b0/dt B + kappa A) T = Q^T B[(2T^n - T^{n-1}/2)/dt + N_T*], lifting 1 - z/Lz;
//   p:  A p = Q^T[sum_a D_a^T (B sum_c dr_a/dx_c f*_c)] - W*, means removed,
//       f* = (2u^n - u^{n-1}/2)/dt + N_u*;
//   u:  (b0/dt B + nu A) u_c = M Q^T[B f*_c - B dp/dx_c];
// BDF2 (3/2, 2, -1/2), EXT2 (2, -1); the first step is BDF1/EXT1 ((1, 1, 0), (1, 0)),
// since BDF2 started from history levels equal to the initial state is first order.
// Explicit terms run in binary64 kernels (double-float for SEM_PREC_DF64);
// the five solves use sem_pcg_solve and the pressure p-multigrid.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <utility>
#include <vector>

#include "sem_fields.cuh"
#include "sem_internal.h"

struct sem_rbc {
  const sem_mesh *m = nullptr;
  sem_rbc_params prm;
  double nu = 0, kappa = 0;
  int step = 0;
  int64_t nL = 0, nU = 0;
  // U-vectors
  double *u[3] = {}, *up[3] = {}, *T = nullptr, *Tp = nullptr, *p = nullptr, *W = nullptr, *Wp = nullptr;
  double *Tb = nullptr, *rhs = nullptr, *x = nullptr, *Tn = nullptr, *un[3] = {};
  double *pp = nullptr;  // p^{n-1}: the second level of the pressure extrapolation
  // u^{n-2}, T^{n-2}: the third level of the third-order guesses (extrapolate = 2 only)
  double *upp[3] = {}, *Tpp = nullptr;
  // E-vectors
  double *uL[3] = {}, *upL[3] = {}, *TL = nullptr, *TpL = nullptr, *g[3] = {}, *om[3] = {};
  double *NT = nullptr, *NTp = nullptr, *Nu[3] = {}, *Nup[3] = {}, *fs[3] = {}, *tmpL = nullptr;
  double *R = nullptr;  // [E][9][n3] dr_a/dx_c
  // double-float split of R; set for SEM_PREC_DF64, where the gradients and
  // the weak divergence run on the binary32 pipe
  float2 *Rdf = nullptr;
  // H Tb = (kappa A + b0/dt B) applied to the lifting (E-vector), kept for the
  // b0/dt it was computed with
  double *HTb = nullptr;
  double keyH = -1.0;
  double *scal = nullptr;  // reduction partials + result
  double *drho = nullptr;  // GLL weights on the device
  int *dnel = nullptr;     // element counts on the device
  void *ws = nullptr;
  size_t ws_bytes = 0;
  sem_pmg *pmg = nullptr;  // pressure preconditioner (pure Neumann hierarchy)
  // Jacobi inverses of the two Helmholtz operators, recomputed only when
  // their coefficients change (the first step's BDF1 b0 differs)
  double *dinvT = nullptr, *dinvU = nullptr;
  double keyT[2] = {-1.0, -1.0}, keyU[2] = {-1.0, -1.0};
  std::vector<void *> owned;
};

namespace {

constexpr int kRedBlocks = 152 * 2;
struct StepCoef {
  double b0, b1, b2, a1, a2;
};
StepCoef coefficients(int step) {
  if (step == 0) return {1.0, 1.0, 0.0, 1.0, 0.0};  // BDF1/EXT1
  return {1.5, 2.0, -0.5, 2.0, -1.0};               // BDF2/EXT2
}

// ---------------------------------------------------------------- kernels
// initial guess x0 = M (2 (a - c) - (b - c)): the extrapolation of the two
// previous levels a = x^n, b = x^{n-1} about the offset c (the lifting of T;
// NULL for none); mask NULL: every node free
__global__ void k_extrap(int64_t n, const uint8_t *__restrict__ mask, const double *__restrict__ a,
                         const double *__restrict__ b, const double *__restrict__ c, double *__restrict__ out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    double v;
    if (c) v = 2.0 * (a[g] - c[g]) - (b[g] - c[g]);
    else v = 2.0 * a[g] - b[g];
    out[g] = (!mask || mask[g]) ? v : 0.0;
  }
}

// third-order guess 3 a - 3 b + d of the levels a = x^n, b = x^{n-1},
// d = x^{n-2} (each less the lifting c when given), zero on masked nodes;
// the operations unfused and in the order the oracle takes them
__global__ void k_extrap3(int64_t n, const uint8_t *__restrict__ mask, const double *__restrict__ a,
                          const double *__restrict__ b, const double *__restrict__ d, const double *__restrict__ c,
                          double *__restrict__ out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    double v;
    if (c) {
      const double cg = c[g];
      v = __dadd_rn(__dsub_rn(__dmul_rn(3.0, __dsub_rn(a[g], cg)), __dmul_rn(3.0, __dsub_rn(b[g], cg))),
                    __dsub_rn(d[g], cg));
    } else {
      v = __dadd_rn(__dsub_rn(__dmul_rn(3.0, a[g]), __dmul_rn(3.0, b[g])), d[g]);
    }
    out[g] = (!mask || mask[g]) ? v : 0.0;
  }
}

// the pressure history: pp <- p; with ex, p <- 2 p - pp (the guess)
__global__ void k_extrap_p(int64_t n, int ex, double *__restrict__ p, double *__restrict__ pp) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const double v = p[g];
    if (ex) p[g] = 2.0 * v - pp[g];
    pp[g] = v;
  }
}

// accumulate the curl of u from grad u_c: om_x = dw/dy - dv/dz, om_y = du/dz - dw/dx, om_z = dv/dx - du/dy
__global__ void k_curl_acc(int64_t nL, int c, const double *__restrict__ g0, const double *__restrict__ g1,
                           const double *__restrict__ g2, double *__restrict__ ox, double *__restrict__ oy,
                           double *__restrict__ oz) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    if (c == 0) {
      ox[l] = 0.0;
      oy[l] = g2[l];
      oz[l] = -g1[l];
    } else if (c == 1) {
      ox[l] -= g2[l];
      oz[l] += g0[l];
    } else {
      ox[l] += g1[l];
      oy[l] -= g0[l];
    }
  }
}

// wall term on one face direction d / side: out_l += nu rho_a rho_b (+-x_a x x_b) . curl(om)
// (elements touching the wall; element-local derivatives of om)
__global__ void k_wall(int n, const int *__restrict__ nel, int d, int side, double nu, const double *__restrict__ D,
                       const double *__restrict__ rho, const double *__restrict__ R, const double *__restrict__ X,
                       const double *__restrict__ Y, const double *__restrict__ Z, const double *__restrict__ ox,
                       const double *__restrict__ oy, const double *__restrict__ oz, double *__restrict__ out) {
  const int n3 = n * n * n, n2 = n * n;
  const int ne[3] = {nel[0], nel[1], nel[2]};
  const int other[2] = {d == 0 ? 1 : 0, d == 2 ? 1 : 2};  // the two element indices across the face
  const int64_t nface_el = (int64_t)ne[other[0]] * ne[other[1]];
  const int64_t total = nface_el * n2;
  const int a = (d + 1) % 3, b = (d + 2) % 3;  // tangential directions with x_a x x_b along +r_d
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t fe = t / n2;
    const int fq = (int)(t - fe * n2);
    int eix[3];
    eix[d] = side ? ne[d] - 1 : 0;
    eix[other[0]] = (int)(fe % ne[other[0]]);
    eix[other[1]] = (int)(fe / ne[other[0]]);
    const int64_t e = eix[0] + (int64_t)ne[0] * (eix[1] + (int64_t)ne[1] * eix[2]);
    int loc[3];
    loc[d] = side ? n - 1 : 0;
    loc[other[0]] = fq % n;
    loc[other[1]] = fq / n;
    const int q = loc[0] + n * (loc[1] + n * loc[2]);
    const int64_t base = e * n3;
    // reference derivatives of om and of the coordinates at this node
    const double *fld[6] = {ox + base, oy + base, oz + base, X + base, Y + base, Z + base};
    double dref[6][3];
    for (int f = 0; f < 6; ++f)
      for (int r = 0; r < 3; ++r) dref[f][r] = 0.0;
    for (int m = 0; m < n; ++m) {
      const int qr = m + n * (loc[1] + n * loc[2]);
      const int qs = loc[0] + n * (m + n * loc[2]);
      const int qt = loc[0] + n * (loc[1] + n * m);
      const double a0 = D[loc[0] * n + m], a1 = D[loc[1] * n + m], a2 = D[loc[2] * n + m];
      for (int f = 0; f < 6; ++f) {
        dref[f][0] = fma(a0, fld[f][qr], dref[f][0]);
        dref[f][1] = fma(a1, fld[f][qs], dref[f][1]);
        dref[f][2] = fma(a2, fld[f][qt], dref[f][2]);
      }
    }
    const double *Re = R + 9 * e * n3 + q;
    double go[3][3];  // go[i][c] = d om_i / d x_c
    for (int i = 0; i < 3; ++i)
      for (int c = 0; c < 3; ++c)
        go[i][c] = Re[(0 + c) * n3] * dref[i][0] + Re[(3 + c) * n3] * dref[i][1] + Re[(6 + c) * n3] * dref[i][2];
    const double cc[3] = {go[2][1] - go[1][2], go[0][2] - go[2][0], go[1][0] - go[0][1]};
    // x_a x x_b from the coordinate derivatives (dref[3 + comp][dir])
    const double xa[3] = {dref[3][a], dref[4][a], dref[5][a]};
    const double xb[3] = {dref[3][b], dref[4][b], dref[5][b]};
    const double area[3] = {xa[1] * xb[2] - xa[2] * xb[1], xa[2] * xb[0] - xa[0] * xb[2], xa[0] * xb[1] - xa[1] * xb[0]};
    const double sgn = side ? 1.0 : -1.0;
    const double wt = rho[loc[a]] * rho[loc[b]];
    out[base + q] += nu * sgn * wt * (area[0] * cc[0] + area[1] * cc[1] + area[2] * cc[2]);
  }
}

// weak divergence: out = sum_a D_a^T v_a with v_a = B sum_c dr_a/dx_c f_c
// Q^T with optional mask: vg[g] = (mask ? mask[g] : 1) * sum of copies
// T right-hand side (local): B ((b1 T + b2 Tp)/dt + a1 NT + a2 NTp) - H(Tb);
// k.b1, k.b2 arrive divided by dt (no division per point)
__global__ void k_rhsT(int64_t nL, StepCoef k, const double *__restrict__ B, const double *__restrict__ TL,
                       const double *__restrict__ TpL, const double *__restrict__ NT, const double *__restrict__ NTp,
                       const double *__restrict__ HTb, double *__restrict__ out) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x)
    out[l] = B[l] * ((k.b1 * TL[l] + k.b2 * TpL[l]) + (k.a1 * NT[l] + k.a2 * NTp[l])) - HTb[l];
}

// f* = (b1 u + b2 up)/dt + a1 Nu + a2 Nup (k.b1, k.b2 divided by dt)
__global__ void k_fstar(int64_t nL, StepCoef k, const double *__restrict__ uL, const double *__restrict__ upL,
                        const double *__restrict__ N, const double *__restrict__ Np, double *__restrict__ out) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x)
    out[l] = (k.b1 * uL[l] + k.b2 * upL[l]) + (k.a1 * N[l] + k.a2 * Np[l]);
}

// B (f - g)
__global__ void k_bdiff(int64_t nL, const double *__restrict__ B, const double *__restrict__ f,
                        const double *__restrict__ g, double *__restrict__ out) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x)
    out[l] = B[l] * (f[l] - g[l]);
}

// y = a x + b y2 + c z (U-vectors; any pointer may alias y)
// fixed-order sum: partials, then one block finishes and stores sum / n// ---------------------------------------------------------------- host helpers
int remove_mean(sem_rbc *s, double *x, cudaStream_t st) {
  k_sum_part<<<kRedBlocks, 256, 0, st>>>(s->nU, x, s->scal);
  k_mean_finish<<<1, 32, 0, st>>>(kRedBlocks, s->nU, s->scal, s->scal + kRedBlocks);
  k_sub_scalar<<<grid_for(s->nU, 256), 256, 0, st>>>(s->nU, s->scal + kRedBlocks, x);
  SEM_LAUNCH_CHECK("remove_mean");
  return SEM_OK;
}

int grad(sem_rbc *s, const double *f, double **out, cudaStream_t st) {
  const sem_mesh *m = s->m;
  if (s->Rdf) return sem_launch_grad_df64(m, s->Rdf, f, out[0], out[1], out[2], st);
  k_grad<<<grid_for(s->nL, 256), 256, 0, st>>>(m->n, m->E, m->dD, s->R, f, out[0], out[1], out[2]);
  SEM_LAUNCH_CHECK("k_grad");
  return SEM_OK;
}

int gather(sem_rbc *s, const double *vL, double *vg, bool masked, cudaStream_t st) {
  const sem_mesh *m = s->m;
  k_gather_m<<<grid_for(s->nU, 256), 256, 0, st>>>(s->nU, m->gs_off, m->gs_perm, masked ? m->mask : nullptr, vL, vg);
  SEM_LAUNCH_CHECK("k_gather_m");
  return SEM_OK;
}

int solve(sem_rbc *s, double h1, double h2, const double *b, double *x, int mask_mode, int guess, int *iters,
          cudaStream_t st, double *dinv = nullptr, double *key = nullptr) {
  sem_solver_opts o;
  o.initial_guess = guess;
  o.tol = s->prm.tol;
  o.maxit = s->prm.maxit;
  o.precision = s->prm.precision;
  o.timeout_s = 0.0;
  o.mask_mode = mask_mode;
  sem_solve_stats stt;
  if (dinv && (key[0] != h1 || key[1] != h2)) {
    if (int rc = sem_jacobi_inv_mode(s->m, h1, h2, mask_mode == 0 ? 1 : 0, dinv, st)) return rc;
    key[0] = h1;
    key[1] = h2;
  }
  int rc = sem_pcg_solve_ex(s->m, h1, h2, b, x, &o, s->ws, &stt, (void *)st, 8, dinv);
  *iters = stt.iterations;
  return rc;
}

void free_rbc(sem_rbc *s) {
  if (!s) return;
  if (s->pmg) sem_pmg_destroy(s->pmg);
  for (void *p : s->owned) cudaFree(p);
  delete s;
}

}  // namespace

extern "C" int sem_rbc_create(const sem_mesh *m, const sem_rbc_params *prm, const double *T_pert_g, void *stream,
                              sem_rbc **out) {
  if (!m || !prm || !out) return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_create: NULL argument");
  *out = nullptr;
  if (m->slab) return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_create: needs the whole box, not a partition's slab mesh");
  if (!(prm->Ra > 0) || !(prm->Pr > 0) || !(prm->dt > 0) || !(prm->tol > 0) || prm->maxit < 1)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_create: Ra, Pr, dt, tol must be > 0 and maxit >= 1");
  if (prm->precision != SEM_PREC_FP64 && prm->precision != SEM_PREC_DF64)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_create: unknown precision");
  if (prm->extrapolate < 0 || prm->extrapolate > 2)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_create: extrapolate must be 0, 1 or 2");
  int dev = -1;
  SEM_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_create: the mesh's device must be current");
  if (m->periodic[2] || !m->dirichlet[4] || !m->dirichlet[5])
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_create: the mesh needs Dirichlet plates at z = 0 and z = Lz");
  if ((!m->periodic[0] && !(m->dirichlet[0] && m->dirichlet[1])) ||
      (!m->periodic[1] && !(m->dirichlet[2] && m->dirichlet[3])))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_create: x and y must be periodic or walls on both sides");
  cudaStream_t st = as_stream(stream);
  sem_rbc *s = new sem_rbc();
  s->m = m;
  s->prm = *prm;
  s->nu = sqrt(prm->Pr / prm->Ra);
  s->kappa = 1.0 / sqrt(prm->Ra * prm->Pr);
  s->nL = m->n_local;
  s->nU = m->n_unique;
  auto alloc = [&](double **p, int64_t count) -> int {
    cudaError_t e = cudaMalloc((void **)p, sizeof(double) * (size_t)std::max<int64_t>(count, 1));
    if (e != cudaSuccess) return sem_cuda_fail(e, "sem_rbc_create: cudaMalloc");
    s->owned.push_back(*p);
    return SEM_OK;
  };
  int rc = SEM_OK;
  double **uvecs[] = {&s->u[0],  &s->u[1], &s->u[2], &s->up[0], &s->up[1], &s->up[2],
                      &s->T,     &s->Tp,   &s->p,    &s->W,     &s->Wp,    &s->Tb,
                      &s->rhs,   &s->x,    &s->Tn,   &s->un[0], &s->un[1], &s->un[2],
                      &s->dinvT, &s->dinvU, &s->pp};
  for (double **p : uvecs)
    if (!rc) rc = alloc(p, s->nU);
  if (prm->extrapolate == 2) {
    double **lv3[] = {&s->upp[0], &s->upp[1], &s->upp[2], &s->Tpp};
    for (double **p : lv3)
      if (!rc) rc = alloc(p, s->nU);
  }
  double **evecs[] = {&s->uL[0], &s->uL[1], &s->uL[2], &s->upL[0], &s->upL[1], &s->upL[2], &s->TL, &s->TpL,
                      &s->g[0],  &s->g[1],  &s->g[2],  &s->om[0],  &s->om[1],  &s->om[2],  &s->NT, &s->NTp,
                      &s->Nu[0], &s->Nu[1], &s->Nu[2], &s->Nup[0], &s->Nup[1], &s->Nup[2], &s->fs[0], &s->fs[1],
                      &s->fs[2], &s->tmpL};
  for (double **p : evecs)
    if (!rc) rc = alloc(p, s->nL);
  if (!rc) rc = alloc(&s->R, 9 * s->nL);
  if (!rc) rc = alloc(&s->HTb, s->nL);
  if (!rc && prm->precision == SEM_PREC_DF64) {
    cudaError_t e = cudaMalloc((void **)&s->Rdf, sizeof(float2) * 9 * (size_t)std::max<int64_t>(s->nL, 1));
    if (e != cudaSuccess) rc = sem_cuda_fail(e, "sem_rbc_create: cudaMalloc(Rdf)");
    else s->owned.push_back(s->Rdf);
  }
  if (!rc) rc = alloc(&s->scal, kRedBlocks + 8);
  if (!rc) rc = alloc(&s->drho, SEM_MAXNP);
  if (!rc) {
    cudaError_t e = cudaMalloc((void **)&s->dnel, sizeof(int) * 3);
    if (e != cudaSuccess) rc = sem_cuda_fail(e, "sem_rbc_create: cudaMalloc");
    else s->owned.push_back(s->dnel);
  }
  if (!rc) rc = sem_pcg_workspace_bytes(m, &s->ws_bytes);
  if (!rc) {
    cudaError_t e = cudaMalloc(&s->ws, s->ws_bytes);
    if (e != cudaSuccess) rc = sem_cuda_fail(e, "sem_rbc_create: cudaMalloc(workspace)");
    else s->owned.push_back(s->ws);
  }
  if (rc) {
    free_rbc(s);
    return rc;
  }
  cudaMemcpyAsync(s->drho, m->rho, sizeof(double) * m->n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(s->dnel, m->nel, sizeof(int) * 3, cudaMemcpyHostToDevice, st);
  k_inv_jacobian<<<grid_for(s->nL, 256), 256, 0, st>>>(m->n, m->E, m->dD, m->X, m->Y, m->Z, s->R);
  if (s->Rdf && (rc = sem_launch_split_df64(s->R, s->Rdf, 9 * s->nL, st))) {
    free_rbc(s);
    return rc;
  }
  k_lifting<<<grid_for(s->nL, 256), 256, 0, st>>>(s->nL, m->L[2], m->l2g, m->Z, s->Tb);
  cudaMemcpyAsync(s->T, s->Tb, sizeof(double) * s->nU, cudaMemcpyDeviceToDevice, st);
  if (T_pert_g) k_add_masked<<<grid_for(s->nU, 256), 256, 0, st>>>(s->nU, m->mask, T_pert_g, s->T);
  // every array a snapshot holds starts defined: u = 0 and zero history
  for (int c = 0; c < 3; ++c) {
    cudaMemsetAsync(s->u[c], 0, sizeof(double) * s->nU, st);
    cudaMemsetAsync(s->up[c], 0, sizeof(double) * s->nU, st);
    cudaMemsetAsync(s->Nup[c], 0, sizeof(double) * s->nL, st);
  }
  cudaMemsetAsync(s->p, 0, sizeof(double) * s->nU, st);
  cudaMemsetAsync(s->pp, 0, sizeof(double) * s->nU, st);
  cudaMemsetAsync(s->Tp, 0, sizeof(double) * s->nU, st);
  cudaMemsetAsync(s->Wp, 0, sizeof(double) * s->nU, st);
  cudaMemsetAsync(s->NTp, 0, sizeof(double) * s->nL, st);
  if (s->Tpp) {
    for (int c = 0; c < 3; ++c) cudaMemsetAsync(s->upp[c], 0, sizeof(double) * s->nU, st);
    cudaMemsetAsync(s->Tpp, 0, sizeof(double) * s->nU, st);
  }
  if (prm->pressure_pmg && m->N > 1) {
    sem_pmg_opts po;
    memset(&po, 0, sizeof(po));
    int c = m->N, nl = 0;
    po.orders[nl++] = c;
    while (c > 1 && nl < 4) {
      c = std::max(1, c / 2);
      po.orders[nl++] = c;
    }
    po.nlevels = nl;
    // geometry of the smoothing levels in bfloat16 (binary32 arithmetic):
    // the same 5 outer iterations as binary32 geometry on the 32^3 RBC mesh,
    // pressure phase 46.3 -> 43.9 ms; the outer FCG stays binary64-accurate
    po.smoother_precision = SEM_PREC_BF16;
    // high-degree 4th-kind Chebyshev: on the plate-stretched elements a
    // degree-2 smoother needs ~30-40 outer iterations, degree 16 about 5, and
    // the whole solve is ~3x faster (measured on the 32^3 RBC mesh)
    po.cheb_degree = 16;
    po.lambda_safety = 1.1;
    po.power_its = 20;
    po.coarse_tol = 1e-2;
    po.coarse_maxit = 2000;
    po.mask_mode = 1;
    if ((rc = sem_pmg_create(m, 1.0, 0.0, &po, stream, &s->pmg))) {
      free_rbc(s);
      return rc;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    rc = sem_cuda_fail(e, "sem_rbc_create: set-up kernels");
    free_rbc(s);
    return rc;
  }
  *out = s;
  return SEM_OK;
}

extern "C" int sem_rbc_destroy(sem_rbc *s) {
  free_rbc(s);
  return SEM_OK;
}

extern "C" int sem_rbc_fields(const sem_rbc *s, sem_rbc_view *v) {
  if (!s || !v) return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_fields: NULL argument");
  v->u = s->u[0];
  v->v = s->u[1];
  v->w = s->u[2];
  v->T = s->T;
  v->p = s->p;
  v->n_unique = s->nU;
  v->step = s->step;
  v->u_prev = s->up[0];
  v->v_prev = s->up[1];
  v->w_prev = s->up[2];
  return SEM_OK;
}

extern "C" int sem_bdf_ext_step(sem_rbc *s, sem_step_stats *stt, void *stream) {
  SemRange nvtx_range("sem_bdf_ext_step");
  if (!s || !stt) return sem_fail(SEM_ERR_INVALID_ARG, "sem_bdf_ext_step: NULL argument");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = as_stream(stream);
  const sem_mesh *m = s->m;
  const int64_t nL = s->nL, nU = s->nU;
  const double dt = s->prm.dt;
  const unsigned gl = grid_for(nL, 256), gu = grid_for(nU, 256);
  int rc;
  stt->status = SEM_OK;
  // level-n fields at the local nodes
  for (int c = 0; c < 3; ++c)
    if ((rc = sem_launch_scatter(m, s->u[c], s->uL[c], st))) return rc;
  if ((rc = sem_launch_scatter(m, s->T, s->TL, st))) return rc;
  // explicit terms: N_T, N_u, curl u, wall term
  if ((rc = grad(s, s->TL, s->g, st))) return rc;
  k_neg_adv<<<gl, 256, 0, st>>>(nL, s->uL[0], s->uL[1], s->uL[2], s->g[0], s->g[1], s->g[2], nullptr, s->NT);
  for (int c = 0; c < 3; ++c) {
    if ((rc = grad(s, s->uL[c], s->g, st))) return rc;
    k_neg_adv<<<gl, 256, 0, st>>>(nL, s->uL[0], s->uL[1], s->uL[2], s->g[0], s->g[1], s->g[2],
                                  c == 2 ? s->TL : nullptr, s->Nu[c]);
    k_curl_acc<<<gl, 256, 0, st>>>(nL, c, s->g[0], s->g[1], s->g[2], s->om[0], s->om[1], s->om[2]);
  }
  SEM_LAUNCH_CHECK("explicit terms");
  SEM_CUDA(cudaMemsetAsync(s->tmpL, 0, sizeof(double) * nL, st));
  for (int d = 0; d < 3; ++d) {  // one launch per wall face: a face writes each of its nodes once
    if (m->periodic[d]) continue;
    for (int side = 0; side < 2; ++side) {
      if (!m->dirichlet[2 * d + side]) continue;
      const int o0 = d == 0 ? 1 : 0, o1 = d == 2 ? 1 : 2;
      const int64_t tot = (int64_t)m->nel[o0] * m->nel[o1] * m->n * m->n;
      k_wall<<<grid_for(tot, 128), 128, 0, st>>>(m->n, s->dnel, d, side, s->nu, m->dD, s->drho, s->R, m->X, m->Y,
                                                 m->Z, s->om[0], s->om[1], s->om[2], s->tmpL);
    }
  }
  SEM_LAUNCH_CHECK("k_wall");
  if ((rc = gather(s, s->tmpL, s->W, false, st))) return rc;
  if (s->step == 0) {  // history = initial state
    for (int c = 0; c < 3; ++c) {
      SEM_CUDA(cudaMemcpyAsync(s->up[c], s->u[c], sizeof(double) * nU, cudaMemcpyDeviceToDevice, st));
      SEM_CUDA(cudaMemcpyAsync(s->Nup[c], s->Nu[c], sizeof(double) * nL, cudaMemcpyDeviceToDevice, st));
    }
    SEM_CUDA(cudaMemcpyAsync(s->Tp, s->T, sizeof(double) * nU, cudaMemcpyDeviceToDevice, st));
    SEM_CUDA(cudaMemcpyAsync(s->NTp, s->NT, sizeof(double) * nL, cudaMemcpyDeviceToDevice, st));
    SEM_CUDA(cudaMemcpyAsync(s->Wp, s->W, sizeof(double) * nU, cudaMemcpyDeviceToDevice, st));
  }
  for (int c = 0; c < 3; ++c)
    if ((rc = sem_launch_scatter(m, s->up[c], s->upL[c], st))) return rc;
  if ((rc = sem_launch_scatter(m, s->Tp, s->TpL, st))) return rc;

  SEM_CUDA(cudaStreamSynchronize(st));
  auto lap = [&, tl = t0]() mutable {
    const auto now = std::chrono::steady_clock::now();
    const double ms = std::chrono::duration<double, std::milli>(now - tl).count();
    tl = now;
    return ms;
  };
  stt->ms_explicit = lap();
  // temperature: lifting Tb, theta = T - Tb on the free nodes
  const StepCoef kc = coefficients(s->step);
  const double b0dt = kc.b0 / dt;
  StepCoef kd = kc;  // b1, b2 divided by dt
  kd.b1 = kc.b1 / dt;
  kd.b2 = kc.b2 / dt;
  if (s->keyH != b0dt) {  // H Tb for this b0/dt (the lifting and kappa are fixed)
    if ((rc = sem_launch_scatter(m, s->Tb, s->fs[0], st))) return rc;
    if ((rc = sem_launch_ax_local(m, s->kappa, b0dt, s->fs[0], s->HTb, s->prm.precision, st))) return rc;
    s->keyH = b0dt;
  }
  k_rhsT<<<gl, 256, 0, st>>>(nL, kd, m->B, s->TL, s->TpL, s->NT, s->NTp, s->HTb, s->tmpL);
  if ((rc = gather(s, s->tmpL, s->rhs, true, st))) return rc;
  // initial guesses: the extrapolation 2 x^n - x^{n-1} once two levels exist;
  // with extrapolate = 2, 3 x^n - 3 x^{n-1} + x^{n-2} for T and u once three do
  const bool ex = s->prm.extrapolate && s->step >= 1;
  const bool ex3 = s->prm.extrapolate == 2 && s->step >= 2;
  if (ex3) {
    k_extrap3<<<gu, 256, 0, st>>>(nU, m->mask, s->T, s->Tp, s->Tpp, s->Tb, s->x);
    SEM_LAUNCH_CHECK("k_extrap3");
  } else if (ex) {
    k_extrap<<<gu, 256, 0, st>>>(nU, m->mask, s->T, s->Tp, s->Tb, s->x);
    SEM_LAUNCH_CHECK("k_extrap");
  }
  rc = solve(s, s->kappa, b0dt, s->rhs, s->x, 0, ex, &stt->iters_T, st, s->dinvT, s->keyT);
  if (rc && rc != SEM_ERR_NOT_CONVERGED) return rc;
  if (rc) stt->status = rc;
  k_axpbypcz<<<gu, 256, 0, st>>>(nU, 1.0, s->Tb, 1.0, s->x, 0.0, nullptr, s->Tn);
  SEM_CUDA(cudaStreamSynchronize(st));
  stt->ms_T = lap();

  // pressure
  for (int c = 0; c < 3; ++c)
    k_fstar<<<gl, 256, 0, st>>>(nL, kd, s->uL[c], s->upL[c], s->Nu[c], s->Nup[c], s->fs[c]);
  if (s->Rdf) {
    if ((rc = sem_launch_wdiv_df64(m, s->Rdf, s->fs[0], s->fs[1], s->fs[2], s->tmpL, st))) return rc;
  } else {
    k_weak_div_v<<<gl, 256, 0, st>>>(m->n, m->E, s->R, m->B, s->fs[0], s->fs[1], s->fs[2], s->g[0], s->g[1],
                                     s->g[2]);
    k_dt_sum<<<gl, 256, 0, st>>>(m->n, m->E, m->dD, s->g[0], s->g[1], s->g[2], s->tmpL);
  }
  SEM_LAUNCH_CHECK("weak divergence");
  if ((rc = gather(s, s->tmpL, s->rhs, false, st))) return rc;
  k_axpbypcz<<<gu, 256, 0, st>>>(nU, 1.0, s->rhs, -kc.a1, s->W, -kc.a2, s->Wp, s->rhs);
  if ((rc = remove_mean(s, s->rhs, st))) return rc;
  // p^{n-1} <- p^n, and p <- 2 p^n - p^{n-1} as the guess when extrapolating
  k_extrap_p<<<gu, 256, 0, st>>>(nU, ex ? 1 : 0, s->p, s->pp);
  SEM_LAUNCH_CHECK("k_extrap_p");
  if (s->pmg) {
    sem_solver_opts o;
    o.initial_guess = ex;
    o.tol = s->prm.tol;
    o.maxit = s->prm.maxit;
    o.precision = s->prm.precision;
    o.timeout_s = 0.0;
    o.mask_mode = 1;
    sem_solve_stats ps;
    rc = sem_pmg_pcg_solve(s->pmg, s->rhs, s->p, &o, &ps, (void *)st);
    stt->iters_p = ps.iterations;
  } else {
    rc = solve(s, 1.0, 0.0, s->rhs, s->p, 1, ex, &stt->iters_p, st);
  }
  if (rc && rc != SEM_ERR_NOT_CONVERGED) return rc;
  if (rc) stt->status = rc;
  if ((rc = remove_mean(s, s->p, st))) return rc;
  SEM_CUDA(cudaStreamSynchronize(st));
  stt->ms_p = lap();

  // velocity
  if ((rc = sem_launch_scatter(m, s->p, s->tmpL, st))) return rc;
  if ((rc = grad(s, s->tmpL, s->g, st))) return rc;
  for (int c = 0; c < 3; ++c) {
    k_bdiff<<<gl, 256, 0, st>>>(nL, m->B, s->fs[c], s->g[c], s->tmpL);
    if ((rc = gather(s, s->tmpL, s->rhs, true, st))) return rc;
    if (ex3) {
      k_extrap3<<<gu, 256, 0, st>>>(nU, m->mask, s->u[c], s->up[c], s->upp[c], nullptr, s->un[c]);
      SEM_LAUNCH_CHECK("k_extrap3");
    } else if (ex) {
      k_extrap<<<gu, 256, 0, st>>>(nU, m->mask, s->u[c], s->up[c], nullptr, s->un[c]);
      SEM_LAUNCH_CHECK("k_extrap");
    }
    rc = solve(s, s->nu, b0dt, s->rhs, s->un[c], 0, ex, &stt->iters_u[c], st, s->dinvU, s->keyU);
    if (rc && rc != SEM_ERR_NOT_CONVERGED) return rc;
    if (rc) stt->status = rc;
  }
  SEM_CUDA(cudaStreamSynchronize(st));
  stt->ms_u = lap();
  // rotate histories (u^{n-2} <- u^{n-1} <- u^n <- u^{n+1}, the same for T)
  for (int c = 0; c < 3; ++c) {
    if (s->Tpp) std::swap(s->upp[c], s->up[c]);
    std::swap(s->up[c], s->u[c]);
    std::swap(s->u[c], s->un[c]);
    std::swap(s->Nup[c], s->Nu[c]);
  }
  if (s->Tpp) std::swap(s->Tpp, s->Tp);
  std::swap(s->Tp, s->T);
  std::swap(s->T, s->Tn);
  std::swap(s->NTp, s->NT);
  std::swap(s->Wp, s->W);
  s->step += 1;
  SEM_CUDA(cudaStreamSynchronize(st));
  stt->step = s->step;
  stt->step_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return stt->status;
}

// ---------------------------------------------------------------- checkpoints
// The state after a step: u, u^{n-1}, T, T^{n-1}, p, W^{n-1}, p^{n-1} (U-vectors),
// with extrapolate = 2 also u^{n-2} and T^{n-2}, then N_T^{n-1}, N_u^{n-1}
// (E-vectors) and the step counter; the rest is rebuilt every step. Layout:
// 64-byte header of eight int64 (step, n_unique, n_local, E, N, format
// version, the bits of dt, 1 when the n-2 levels are held else 0) then the
// arrays in that order.
namespace {

struct StateLayout {
  std::vector<std::pair<double *, int64_t>> arrays;
  size_t bytes;
};

StateLayout layout(const sem_rbc *s) {
  StateLayout L;
  double *uvec[] = {s->u[0], s->u[1], s->u[2], s->up[0], s->up[1], s->up[2], s->T, s->Tp, s->p, s->Wp, s->pp};
  for (double *p : uvec) L.arrays.push_back({p, s->nU});
  if (s->Tpp) {  // the third levels of the third-order guesses
    double *lv3[] = {s->upp[0], s->upp[1], s->upp[2], s->Tpp};
    for (double *p : lv3) L.arrays.push_back({p, s->nU});
  }
  double *evec[] = {s->NTp, s->Nup[0], s->Nup[1], s->Nup[2]};
  for (double *p : evec) L.arrays.push_back({p, s->nL});
  L.bytes = 64;
  for (auto &a : L.arrays) L.bytes += sizeof(double) * (size_t)a.second;
  return L;
}

constexpr int64_t kStateVersion = 2;  // 2: p^{n-1} added

void make_header(const sem_rbc *s, int64_t hdr[8]) {
  int64_t dtbits;
  memcpy(&dtbits, &s->prm.dt, sizeof(dtbits));
  const int64_t h[8] = {s->step, s->nU, s->nL, s->m->E, s->m->N, kStateVersion, dtbits, s->Tpp ? 1 : 0};
  memcpy(hdr, h, sizeof(h));
}

// a header fits this state if everything but the step counter matches
bool header_fits(const sem_rbc *s, const int64_t hdr[8]) {
  int64_t mine[8];
  make_header(s, mine);
  return hdr[0] >= 0 && hdr[0] <= INT32_MAX && memcmp(hdr + 1, mine + 1, 7 * sizeof(int64_t)) == 0;
}

uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t h) {
  for (size_t t = 0; t < n; ++t) h = (h ^ p[t]) * 1099511628211ull;
  return h;
}

}  // namespace

extern "C" int sem_rbc_state_bytes(const sem_rbc *s, size_t *bytes) {
  if (!s || !bytes) return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_state_bytes: NULL argument");
  *bytes = layout(s).bytes;
  return SEM_OK;
}

extern "C" int sem_rbc_save_state(const sem_rbc *s, void *dev_buf, void *stream) {
  if (!s || !dev_buf) return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_save_state: NULL argument");
  cudaStream_t st = as_stream(stream);
  int64_t hdr[8];
  make_header(s, hdr);
  SEM_CUDA(cudaMemcpyAsync(dev_buf, hdr, sizeof(hdr), cudaMemcpyHostToDevice, st));
  size_t off = 64;
  for (auto &a : layout(s).arrays) {
    SEM_CUDA(cudaMemcpyAsync((char *)dev_buf + off, a.first, sizeof(double) * a.second, cudaMemcpyDeviceToDevice, st));
    off += sizeof(double) * a.second;
  }
  SEM_CUDA(cudaStreamSynchronize(st));  // the header lives on this stack frame
  return SEM_OK;
}

extern "C" int sem_rbc_load_state(sem_rbc *s, const void *dev_buf, void *stream) {
  if (!s || !dev_buf) return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_load_state: NULL argument");
  cudaStream_t st = as_stream(stream);
  int64_t hdr[8];
  SEM_CUDA(cudaMemcpyAsync(hdr, dev_buf, sizeof(hdr), cudaMemcpyDeviceToHost, st));
  SEM_CUDA(cudaStreamSynchronize(st));
  if (!header_fits(s, hdr))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_load_state: the snapshot belongs to another mesh, dt or format");
  size_t off = 64;
  for (auto &a : layout(s).arrays) {
    SEM_CUDA(cudaMemcpyAsync(a.first, (const char *)dev_buf + off, sizeof(double) * a.second,
                             cudaMemcpyDeviceToDevice, st));
    off += sizeof(double) * a.second;
  }
  SEM_CUDA(cudaStreamSynchronize(st));
  s->step = (int)hdr[0];
  return SEM_OK;
}

// File checkpoint: magic "SEMRBC01", the state header and arrays, then an
// FNV-1a 64-bit checksum of everything before it.
extern "C" int sem_rbc_save(const sem_rbc *s, const char *path) {
  if (!s || !path) return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_save: NULL argument");
  const StateLayout L = layout(s);
  std::vector<unsigned char> buf(8 + L.bytes);
  memcpy(buf.data(), "SEMRBC01", 8);
  int64_t hdr[8];
  make_header(s, hdr);
  memcpy(buf.data() + 8, hdr, 64);
  size_t off = 8 + 64;
  for (auto &a : L.arrays) {
    SEM_CUDA(cudaMemcpy(buf.data() + off, a.first, sizeof(double) * a.second, cudaMemcpyDeviceToHost));
    off += sizeof(double) * a.second;
  }
  const uint64_t h = fnv1a(buf.data(), buf.size(), 1469598103934665603ull);
  FILE *f = fopen(path, "wb");
  if (!f) return sem_fail(SEM_ERR_IO, std::string("sem_rbc_save: cannot open ") + path);
  const bool ok = fwrite(buf.data(), 1, buf.size(), f) == buf.size() && fwrite(&h, sizeof(h), 1, f) == 1;
  if (fclose(f) != 0 || !ok) return sem_fail(SEM_ERR_IO, std::string("sem_rbc_save: write failed: ") + path);
  return SEM_OK;
}

extern "C" int sem_rbc_load(sem_rbc *s, const char *path) {
  if (!s || !path) return sem_fail(SEM_ERR_INVALID_ARG, "sem_rbc_load: NULL argument");
  const StateLayout L = layout(s);
  std::vector<unsigned char> buf(8 + L.bytes);
  uint64_t h = 0;
  FILE *f = fopen(path, "rb");
  if (!f) return sem_fail(SEM_ERR_IO, std::string("sem_rbc_load: cannot open ") + path);
  const bool ok = fread(buf.data(), 1, buf.size(), f) == buf.size() && fread(&h, sizeof(h), 1, f) == 1;
  fclose(f);
  if (!ok) return sem_fail(SEM_ERR_IO, "sem_rbc_load: file truncated or of another mesh");
  if (memcmp(buf.data(), "SEMRBC01", 8) != 0) return sem_fail(SEM_ERR_IO, "sem_rbc_load: not a checkpoint");
  if (fnv1a(buf.data(), buf.size(), 1469598103934665603ull) != h) return sem_fail(SEM_ERR_IO, "sem_rbc_load: checksum mismatch");
  int64_t hdr[8];
  memcpy(hdr, buf.data() + 8, 64);
  if (!header_fits(s, hdr)) return sem_fail(SEM_ERR_IO, "sem_rbc_load: checkpoint of another mesh, dt or format");
  size_t off = 8 + 64;
  for (auto &a : L.arrays) {
    SEM_CUDA(cudaMemcpy(a.first, buf.data() + off, sizeof(double) * a.second, cudaMemcpyHostToDevice));
    off += sizeof(double) * a.second;
  }
  s->step = (int)hdr[0];
  return SEM_OK;
}
