// Operator entry points of the C ABI and the Jacobi-preconditioned conjugate
// gradient solve of the assembled Helmholtz system (Sec. 2.2: the pressure
// Poisson solve is the stiffest substep and is preconditioned).
//
// Vectors are U-vectors (one value per unique node). Each iteration runs
//   w = M Q^T A_L Q p  (fused operator into w = 0, also the p.w partial sums)
//   update1: alpha = rho / p.w;  x += alpha p;  r -= alpha w;  partial r.z, r.r
//   update2: beta = r.z / rho;   p = z + beta p   (z = dinv * r, not stored);
//            w = 0 for the next operator; the stopping test on the device
// (On GB300 binary64 arithmetic runs at 1/64 of the binary32 rate, so these
// streaming kernels are bound by memory or by the FP64 pipe: update1 does
// five binary64 operations per node against seven vector words, update2 two
// against five. With x += alpha p in update2 instead, update1's four
// operations against four words made it FP64-bound, 0.44 of DRAM
// throughput, and the pair was slower although it moved one word less.)
// All reductions are two-level and in a fixed order, so for a given mesh and
// input every scalar is reproducible except through the operator's atomics.
// The stopping test (||r|| <= tol ||b||, or a breakdown) is taken by update2
// itself, which records the iteration in the scalars; the kernels of later
// iterations then return at once. The host can therefore queue several
// iterations between reads of the scalars and still stop exactly where a
// check after every iteration would.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <mutex>
#include <string>

#include <cuda.h>

#include "sem_internal.h"

namespace {

constexpr int kUpdThreads = 256;
constexpr int kCheckEvery = 8;  // iterations queued between host reads of the scalars
constexpr int kUpdBlocks = 152 * 4;

struct PcgScalars {
  double rho[2];  // r.z, ping-pong by iteration parity
  double pw;      // p.w of the last iteration
  double alpha;
  double beta;
  double rr;      // r.r after the last update
  double bb;      // b.b
  int stop_it;    // 0 while running; else the iteration at which the solve stopped
  int stop_status;  // 1: converged, 2: breakdown (written before stop_it)
};

__device__ __forceinline__ double block_sum(double v, double *red) {
  // fixed-order block reduction; red must hold 32 doubles; result in all threads
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// every block sums the same partial array in the same order
__device__ __forceinline__ double sum_partials(const double *__restrict__ part, int n, double *red) {
  double v = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) v += part[t];
  return block_sum(v, red);
}

__global__ void __launch_bounds__(kUpdThreads)
    k_pcg_init(int64_t nU, const double *__restrict__ b, double inv_scale, double *__restrict__ x,
               double *__restrict__ r, double *__restrict__ p, double *__restrict__ w,
               const double *__restrict__ dinv, double *__restrict__ part_a, double *__restrict__ part_b) {
  __shared__ double red[32];
  double rz = 0.0, bb = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nU; g += (int64_t)gridDim.x * blockDim.x) {
    const double bv = b[g] * inv_scale;
    const double z = dinv[g] * bv;
    x[g] = 0.0;
    r[g] = bv;
    p[g] = z;
    w[g] = 0.0;
    rz = fma(bv, z, rz);
    bb = fma(bv, bv, bb);
  }
  rz = block_sum(rz, red);
  bb = block_sum(bb, red);
  if (threadIdx.x == 0) {
    part_a[blockIdx.x] = rz;
    part_b[blockIdx.x] = bb;
  }
}

// start from an initial guess: x holds the (scaled) guess and w = A x on
// entry; r = b - A x, p = z = dinv r, w = 0 for the first operator
__global__ void __launch_bounds__(kUpdThreads)
    k_pcg_init_guess(int64_t nU, const double *__restrict__ b, double inv_scale, double *__restrict__ r,
                     double *__restrict__ p, double *__restrict__ w, const double *__restrict__ dinv,
                     double *__restrict__ part_a, double *__restrict__ part_b, double *__restrict__ part_c) {
  __shared__ double red[32];
  double rz = 0.0, bb = 0.0, rr = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nU; g += (int64_t)gridDim.x * blockDim.x) {
    const double bv = b[g] * inv_scale;
    const double rv = bv - w[g];
    const double z = dinv[g] * rv;
    r[g] = rv;
    p[g] = z;
    w[g] = 0.0;
    rz = fma(rv, z, rz);
    bb = fma(bv, bv, bb);
    rr = fma(rv, rv, rr);
  }
  rz = block_sum(rz, red);
  bb = block_sum(bb, red);
  rr = block_sum(rr, red);
  if (threadIdx.x == 0) {
    part_a[blockIdx.x] = rz;
    part_b[blockIdx.x] = bb;
    part_c[blockIdx.x] = rr;
  }
}

// part_c: the r.r partials when the solve starts from a guess; NULL when r = b
__global__ void __launch_bounds__(kUpdThreads)
    k_pcg_init_finish(const double *__restrict__ part_a, const double *__restrict__ part_b,
                      const double *__restrict__ part_c, int n, PcgScalars *s) {
  __shared__ double red[32];
  const double rz = sum_partials(part_a, n, red);
  const double bb = sum_partials(part_b, n, red);
  const double rr = part_c ? sum_partials(part_c, n, red) : bb;
  if (threadIdx.x == 0) {
    s->rho[0] = rz;
    s->bb = bb;
    s->rr = rr;
    s->stop_it = 0;
    s->stop_status = 0;
  }
}

// The operator leaves up to hundreds of thousands of p.w partials (one per
// warp of the double-float operator). Block b of this kernel sums the chunk
// [b chunk, (b + 1) chunk) in a fixed order, and every update1 CTA then sums
// the (at most kUpdBlocks) chunk sums in the same order: a fixed-order
// two-level sum (one CTA summing 4 MB of partials took 0.24 ms per iteration
// on 64^3).
constexpr int kPwChunk = 1024;  // the chunk length, raised for meshes with more than kUpdBlocks chunks
__global__ void __launch_bounds__(kUpdThreads)
    k_pw_reduce(const double *__restrict__ pw_part, int n_pw, int chunk, double *__restrict__ out,
                const PcgScalars *s) {
  __shared__ double red[32];
  if (*(volatile const int *)&s->stop_it != 0) return;  // stopped at an earlier iteration
  const int b0 = blockIdx.x * chunk;
  const int n = min(chunk, n_pw - b0);
  const double v = sum_partials(pw_part + b0, n, red);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kUpdThreads)
    k_pcg_update1(int64_t nU, double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                  const double *__restrict__ w, const double *__restrict__ dinv, const double *__restrict__ pw_part,
                  int n_pw, PcgScalars *s, int par, double *__restrict__ rz_part, double *__restrict__ rr_part) {
  __shared__ double red[32];
  if (*(volatile const int *)&s->stop_it != 0) return;  // stopped at an earlier iteration
  const double pw = sum_partials(pw_part, n_pw, red);
  // an exactly converged iterate (p = 0) gives p.w = 0: take no step; the host
  // reports a breakdown only if the residual has not met the tolerance
  const double alpha = (pw > 0.0) ? s->rho[par] / pw : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s->pw = pw;
    s->alpha = alpha;
  }
  double rz = 0.0, rr = 0.0;
  // The grid-stride loop takes four nodes per pass with all their loads
  // issued first (enough loads in flight to cover the memory latency with
  // 608 CTAs); each thread still visits its nodes in the plain loop's order,
  // so the partial sums are the same bits.
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; g + 3 * S < nU; g += 4 * S) {
    double pv[4], xv[4], wv[4], rv0[4], dv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      pv[u] = p[g + u * S];
      xv[u] = x[g + u * S];
      wv[u] = w[g + u * S];
      rv0[u] = r[g + u * S];
      dv[u] = dinv[g + u * S];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x[g + u * S] = fma(alpha, pv[u], xv[u]);
      const double rv = fma(-alpha, wv[u], rv0[u]);
      r[g + u * S] = rv;
      const double z = dv[u] * rv;
      rz = fma(rv, z, rz);
      rr = fma(rv, rv, rr);
    }
  }
  for (; g < nU; g += S) {
    x[g] = fma(alpha, p[g], x[g]);
    const double rv = fma(-alpha, w[g], r[g]);
    r[g] = rv;
    const double z = dinv[g] * rv;
    rz = fma(rv, z, rz);
    rr = fma(rv, rv, rr);
  }
  rz = block_sum(rz, red);
  rr = block_sum(rr, red);
  if (threadIdx.x == 0) {
    rz_part[blockIdx.x] = rz;
    rr_part[blockIdx.x] = rr;
  }
}

__global__ void __launch_bounds__(kUpdThreads)
    k_pcg_update2(int64_t nU, const double *__restrict__ r, double *__restrict__ p, double *__restrict__ w,
                  const double *__restrict__ dinv, const double *__restrict__ rz_part,
                  const double *__restrict__ rr_part, int n_part, PcgScalars *s, int par, int it, double thresh) {
  __shared__ double red[32];
  // block 0 of this launch may record a stop at this iteration while the other
  // blocks read the flag; only a stop at an earlier iteration skips the work
  const int sit = *(volatile const int *)&s->stop_it;
  if (sit != 0 && sit < it) return;
  const double rz = sum_partials(rz_part, n_part, red);
  const double rho_old = s->rho[par];
  const double beta = (rho_old != 0.0) ? rz / rho_old : 0.0;
  if (blockIdx.x == 0) {  // only block 0 needs r.r (block-uniform branch)
    const double rr = sum_partials(rr_part, n_part, red);
    if (threadIdx.x == 0) {
      s->rr = rr;
      s->beta = beta;
      s->rho[par ^ 1] = rz;
      const double pw = s->pw;
      int status = 0;
      if (isfinite(rr) && sqrt(rr) <= thresh) status = 1;
      else if (!(pw > 0.0) || !isfinite(pw) || !isfinite(rr)) status = 2;
      if (status != 0) {
        s->stop_status = status;
        __threadfence();
        *(volatile int *)&s->stop_it = it;
      }
    }
  }
  // four nodes per pass, loads first (as in k_pcg_update1)
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; g + 3 * S < nU; g += 4 * S) {
    double pv[4], rv[4], dv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      pv[u] = p[g + u * S];
      rv[u] = r[g + u * S];
      dv[u] = dinv[g + u * S];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      p[g + u * S] = fma(beta, pv[u], dv[u] * rv[u]);
      w[g + u * S] = 0.0;
    }
  }
  for (; g < nU; g += S) {
    p[g] = fma(beta, p[g], dinv[g] * r[g]);
    w[g] = 0.0;
  }
}

// partial sums of b.b (for the scale of the system)
__global__ void __launch_bounds__(kUpdThreads)
    k_norm2_part(int64_t nU, const double *__restrict__ b, double *__restrict__ part) {
  __shared__ double red[32];
  double bb = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nU; g += (int64_t)gridDim.x * blockDim.x)
    bb = fma(b[g], b[g], bb);
  bb = block_sum(bb, red);
  if (threadIdx.x == 0) part[blockIdx.x] = bb;
}

__global__ void __launch_bounds__(kUpdThreads)
    k_sum_finish(const double *__restrict__ part, int n, PcgScalars *s) {
  __shared__ double red[32];
  const double v = sum_partials(part, n, red);
  if (threadIdx.x == 0) s->bb = v;
}

__global__ void k_scale(int64_t n, double a, double *__restrict__ x) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    x[g] *= a;
}

// dinv[g] = mask[g] / sum over copies of the local diagonal
__global__ void k_jacobi_inv(int n, int64_t nU, const int32_t *__restrict__ off, const int32_t *__restrict__ perm,
                             const uint8_t *__restrict__ mask, const double *__restrict__ Dg,
                             const double *__restrict__ G, const double *__restrict__ B, double h1, double h2,
                             int use_mask, double *__restrict__ dinv) {
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
    dinv[g] = (!use_mask || mask[g]) ? 1.0 / tot : 0.0;
  }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct PcgWork {
  double *r, *p, *w, *dinv, *pw_part, *part_a, *part_b, *part_c;
  PcgScalars *s;
};

size_t pcg_layout(const sem_mesh *m, char *base, PcgWork *wk) {
  const size_t vec = align256(sizeof(double) * (size_t)m->n_unique);
  const size_t npw = align256(sizeof(double) * (size_t)std::max(sem_ax_assembled_blocks(m, SEM_PREC_FP64),
                                                                 sem_ax_assembled_blocks(m, SEM_PREC_DF64)));
  const size_t npart = align256(sizeof(double) * kUpdBlocks);
  size_t off = 0;
  auto take = [&](size_t b) {
    char *p = base ? base + off : nullptr;
    off += b;
    return p;
  };
  PcgWork w;
  w.r = (double *)take(vec);
  w.p = (double *)take(vec);
  w.w = (double *)take(vec);
  w.dinv = (double *)take(vec);
  w.pw_part = (double *)take(npw);
  w.part_a = (double *)take(npart);
  w.part_b = (double *)take(npart);
  w.part_c = (double *)take(npart);
  w.s = (PcgScalars *)take(align256(sizeof(PcgScalars)));
  if (wk) *wk = w;
  return off;
}

int check_mesh(const sem_mesh *m, const char *fn) {
  if (!m) return sem_fail(SEM_ERR_INVALID_ARG, std::string(fn) + ": NULL mesh");
  return SEM_OK;
}

bool bad_ptr(const void *p) { return p == nullptr || ((uintptr_t)p & 7) != 0; }

}  // namespace

extern "C" int sem_ax_apply(const sem_mesh *m, double h1, double h2, const double *u_L, double *w_L, int precision,
                            void *stream) {
  SemRange nvtx_range("sem_ax_apply");
  if (int rc = check_mesh(m, "sem_ax_apply")) return rc;
  if (bad_ptr(u_L) || bad_ptr(w_L)) return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_apply: NULL or misaligned vector");
  if (u_L == w_L) return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_apply: u_L and w_L must not overlap");
  if (precision != SEM_PREC_FP64 && precision != SEM_PREC_DF64)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_apply: unknown precision");
  return sem_launch_ax_local(m, h1, h2, u_L, w_L, precision, as_stream(stream));
}

extern "C" int sem_gs_op(const sem_mesh *m, double *v_L, int apply_mask, void *stream) {
  SemRange nvtx_range("sem_gs_op");
  if (int rc = check_mesh(m, "sem_gs_op")) return rc;
  if (bad_ptr(v_L)) return sem_fail(SEM_ERR_INVALID_ARG, "sem_gs_op: NULL or misaligned vector");
  return sem_launch_gs(m, v_L, apply_mask, as_stream(stream));
}

extern "C" int sem_gather(const sem_mesh *m, const double *v_L, double *v_g, void *stream) {
  if (int rc = check_mesh(m, "sem_gather")) return rc;
  if (bad_ptr(v_L) || bad_ptr(v_g)) return sem_fail(SEM_ERR_INVALID_ARG, "sem_gather: NULL or misaligned vector");
  return sem_launch_gather(m, v_L, v_g, as_stream(stream));
}

extern "C" int sem_scatter(const sem_mesh *m, const double *v_g, double *v_L, void *stream) {
  if (int rc = check_mesh(m, "sem_scatter")) return rc;
  if (bad_ptr(v_L) || bad_ptr(v_g)) return sem_fail(SEM_ERR_INVALID_ARG, "sem_scatter: NULL or misaligned vector");
  return sem_launch_scatter(m, v_g, v_L, as_stream(stream));
}

extern "C" int sem_ax_assembled(const sem_mesh *m, double h1, double h2, const double *u_g, double *w_g, int precision,
                                void *stream) {
  SemRange nvtx_range("sem_ax_assembled");
  if (int rc = check_mesh(m, "sem_ax_assembled")) return rc;
  if (bad_ptr(u_g) || bad_ptr(w_g)) return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled: NULL or misaligned vector");
  if (u_g == w_g) return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled: u_g and w_g must not overlap");
  if (precision != SEM_PREC_FP64 && precision != SEM_PREC_DF64)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled: unknown precision");
  cudaStream_t st = as_stream(stream);
  SEM_CUDA(cudaMemsetAsync(w_g, 0, sizeof(double) * m->n_unique, st));
  return sem_launch_ax_assembled(m, h1, h2, u_g, w_g, nullptr, precision, st);
}

extern "C" int sem_ax_assembled_add(const sem_mesh *m, double h1, double h2, const double *u_g, double *w_g,
                                    int precision, void *stream) {
  if (int rc = check_mesh(m, "sem_ax_assembled_add")) return rc;
  if (bad_ptr(u_g) || bad_ptr(w_g)) return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_add: NULL or misaligned vector");
  if (u_g == w_g) return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_add: u_g and w_g must not overlap");
  if (precision != SEM_PREC_FP64 && precision != SEM_PREC_DF64)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_add: unknown precision");
  return sem_launch_ax_assembled(m, h1, h2, u_g, w_g, nullptr, precision, as_stream(stream));
}

extern "C" int sem_jacobi_inv(const sem_mesh *m, double h1, double h2, double *dinv_g, void *stream) {
  if (int rc = check_mesh(m, "sem_jacobi_inv")) return rc;
  if (bad_ptr(dinv_g)) return sem_fail(SEM_ERR_INVALID_ARG, "sem_jacobi_inv: NULL or misaligned vector");
  k_jacobi_inv<<<grid_for(m->n_unique, 256), 256, 0, as_stream(stream)>>>(
      m->n, m->n_unique, m->gs_off, m->gs_perm, m->mask, m->dD, m->G, m->B, h1, h2, 1, dinv_g);
  SEM_LAUNCH_CHECK("k_jacobi_inv");
  return SEM_OK;
}

int sem_jacobi_inv_mode(const sem_mesh *m, double h1, double h2, int use_mask, double *dinv_g, cudaStream_t st) {
  k_jacobi_inv<<<grid_for(m->n_unique, 256), 256, 0, st>>>(m->n, m->n_unique, m->gs_off, m->gs_perm, m->mask, m->dD,
                                                            m->G, m->B, h1, h2, use_mask, dinv_g);
  SEM_LAUNCH_CHECK("k_jacobi_inv");
  return SEM_OK;
}

extern "C" int sem_pcg_workspace_bytes(const sem_mesh *m, size_t *bytes) {
  if (int rc = check_mesh(m, "sem_pcg_workspace_bytes")) return rc;
  if (!bytes) return sem_fail(SEM_ERR_INVALID_ARG, "sem_pcg_workspace_bytes: NULL output");
  *bytes = pcg_layout(m, nullptr, nullptr);
  return SEM_OK;
}

extern "C" int sem_pcg_solve(const sem_mesh *m, double h1, double h2, const double *b_g, double *x_g,
                             const sem_solver_opts *opts, void *workspace, sem_solve_stats *stats, void *stream) {
  return sem_pcg_solve_ex(m, h1, h2, b_g, x_g, opts, workspace, stats, stream, kCheckEvery);
}

// check_every: the host reads the scalars (stop flag, timeout) only every
// check_every iterations; the step lengths and the stopping test are computed
// on the device, so the result does not depend on it (iterations queued past
// the stop return at once).
int sem_pcg_solve_ex(const sem_mesh *m, double h1, double h2, const double *b_g, double *x_g,
                     const sem_solver_opts *opts, void *workspace, sem_solve_stats *stats, void *stream,
                     int check_every, const double *dinv_given) {
  SemRange nvtx_range("sem_pcg_solve_ex");
  if (int rc = check_mesh(m, "sem_pcg_solve")) return rc;
  if (check_every < 1) check_every = 1;
  if (bad_ptr(b_g) || bad_ptr(x_g)) return sem_fail(SEM_ERR_INVALID_ARG, "sem_pcg_solve: NULL or misaligned vector");
  if (!opts || !stats) return sem_fail(SEM_ERR_INVALID_ARG, "sem_pcg_solve: NULL opts or stats");
  if (!workspace || ((uintptr_t)workspace & 255))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pcg_solve: workspace must be non-NULL and 256-byte aligned");
  if (!(opts->tol >= 0.0) || opts->maxit < 1) return sem_fail(SEM_ERR_INVALID_ARG, "sem_pcg_solve: bad tol or maxit");
  if (opts->precision != SEM_PREC_FP64 && opts->precision != SEM_PREC_DF64)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pcg_solve: unknown precision");
  if (opts->mask_mode != 0 && opts->mask_mode != 1) return sem_fail(SEM_ERR_INVALID_ARG, "sem_pcg_solve: bad mask_mode");
  if (opts->initial_guess != 0 && opts->initial_guess != 1)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pcg_solve: initial_guess must be 0 or 1");
  if (!(h1 >= 0.0) || !(h2 >= 0.0) || (h1 == 0.0 && h2 == 0.0))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pcg_solve: need h1 >= 0, h2 >= 0, not both zero");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = as_stream(stream);
  PcgWork wk;
  pcg_layout(m, (char *)workspace, &wk);
  const int n_pw = sem_ax_assembled_blocks(m, opts->precision);
  // update kernels: no more CTAs than the vector needs (each CTA re-sums the
  // partials of the previous kernel, so fewer CTAs also means less of that)
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(kUpdBlocks, (m->n_unique + 2047) / 2048));
  const int64_t nU = m->n_unique;
  stats->iterations = 0;
  stats->rel_residual = 0.0;
  stats->solve_ms = 0.0;
  stats->status = SEM_OK;

  int rc;
  const bool masked = opts->mask_mode == 0;
  const int32_t *map = masked ? m->l2gm : m->l2g;
  const double *dinv = dinv_given ? dinv_given : wk.dinv;
  if (!dinv_given) {
    k_jacobi_inv<<<grid_for(m->n_unique, 256), 256, 0, st>>>(m->n, m->n_unique, m->gs_off, m->gs_perm, m->mask,
                                                              m->dD, m->G, m->B, h1, h2, masked ? 1 : 0, wk.dinv);
    SEM_LAUNCH_CHECK("k_jacobi_inv");
  }
  // Solve the system scaled by an exact power of two so that ||b|| ~ 1: the
  // iteration is unchanged in binary64 (power-of-two scaling is exact) and
  // the double-float operator stays inside the binary32 exponent range.
  PcgScalars hs;
  k_norm2_part<<<kUpdBlocks, kUpdThreads, 0, st>>>(nU, b_g, wk.part_a);
  k_sum_finish<<<1, kUpdThreads, 0, st>>>(wk.part_a, kUpdBlocks, wk.s);
  SEM_LAUNCH_CHECK("k_norm2_part");
  SEM_CUDA(cudaMemcpyAsync(&hs, wk.s, sizeof(hs), cudaMemcpyDeviceToHost, st));
  SEM_CUDA(cudaStreamSynchronize(st));
  double scale = 1.0;
  if (hs.bb > 0.0 && std::isfinite(hs.bb)) scale = std::ldexp(1.0, std::ilogb(sqrt(hs.bb)));
  // a guess is used only for a finite, nonzero b (b = 0 gives x = 0)
  const bool guess = opts->initial_guess == 1 && hs.bb > 0.0 && std::isfinite(hs.bb);
  if (guess) {  // x <- x / scale (exact), w = A x, r = b / scale - w
    k_scale<<<grid_for(nU, 256), 256, 0, st>>>(nU, 1.0 / scale, x_g);
    SEM_CUDA(cudaMemsetAsync(wk.w, 0, sizeof(double) * nU, st));
    if ((rc = sem_launch_ax_assembled(m, h1, h2, x_g, wk.w, nullptr, opts->precision, st, map)) != SEM_OK) return rc;
    k_pcg_init_guess<<<kUpdBlocks, kUpdThreads, 0, st>>>(nU, b_g, 1.0 / scale, wk.r, wk.p, wk.w, dinv, wk.part_a,
                                                         wk.part_b, wk.part_c);
  } else {
    k_pcg_init<<<kUpdBlocks, kUpdThreads, 0, st>>>(nU, b_g, 1.0 / scale, x_g, wk.r, wk.p, wk.w, dinv, wk.part_a,
                                                   wk.part_b);
  }
  k_pcg_init_finish<<<1, kUpdThreads, 0, st>>>(wk.part_a, wk.part_b, guess ? wk.part_c : nullptr, kUpdBlocks, wk.s);
  SEM_LAUNCH_CHECK("k_pcg_init");
  SEM_CUDA(cudaMemcpyAsync(&hs, wk.s, sizeof(hs), cudaMemcpyDeviceToHost, st));
  SEM_CUDA(cudaStreamSynchronize(st));
  const double bnorm = sqrt(hs.bb);
  auto finish = [&](int status, int it, double rr) {
    if (scale != 1.0 && (it > 0 || guess)) {
      // undo the scaling of x; if that fails, x is not the solution and the
      // call reports the CUDA error instead of the solver status
      k_scale<<<grid_for(nU, 256), 256, 0, st>>>(nU, scale, x_g);
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) status = sem_cuda_fail(e, "sem_pcg_solve: rescaling the solution");
    }
    stats->iterations = it;
    stats->rel_residual = (bnorm > 0.0) ? sqrt(rr) / bnorm : 0.0;
    stats->solve_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    stats->status = status;
    if (status == SEM_ERR_NOT_CONVERGED) sem_fail(status, "sem_pcg_solve: maxit reached");
    if (status == SEM_ERR_BREAKDOWN) sem_fail(status, "sem_pcg_solve: breakdown (p.Ap <= 0 or non-finite)");
    if (status == SEM_ERR_TIMEOUT) sem_fail(status, "sem_pcg_solve: timeout");
    return status;
  };
  if (!(bnorm > 0.0)) {
    if (!std::isfinite(hs.bb)) return finish(SEM_ERR_BREAKDOWN, 0, hs.bb);
    return finish(SEM_OK, 0, 0.0);  // b = 0: x = 0 (already written)
  }
  const double thresh = opts->tol * bnorm;
  // p.w chunks: at most kUpdBlocks of them (the size of part_c)
  const int chunk = std::max(kPwChunk, (n_pw + kUpdBlocks - 1) / kUpdBlocks);
  const int n_chunks = std::max(1, (n_pw + chunk - 1) / chunk);
  if (guess) {  // the guess may already meet the tolerance, or be non-finite
    if (!std::isfinite(hs.rr) || !std::isfinite(hs.rho[0])) return finish(SEM_ERR_BREAKDOWN, 0, hs.rr);
    if (sqrt(hs.rr) <= thresh) return finish(SEM_OK, 0, hs.rr);
  }
  const int *stop = &wk.s->stop_it;
  for (int it = 1; it <= opts->maxit; ++it) {
    const int par = (it - 1) & 1;
    if ((rc = sem_launch_ax_assembled(m, h1, h2, wk.p, wk.w, wk.pw_part, opts->precision, st, map, stop)) != SEM_OK)
      return rc;
    k_pw_reduce<<<n_chunks, kUpdThreads, 0, st>>>(wk.pw_part, n_pw, chunk, wk.part_c, wk.s);
    k_pcg_update1<<<nblk, kUpdThreads, 0, st>>>(nU, x_g, wk.r, wk.p, wk.w, dinv, wk.part_c, n_chunks, wk.s, par,
                                                wk.part_a, wk.part_b);
    k_pcg_update2<<<nblk, kUpdThreads, 0, st>>>(nU, wk.r, wk.p, wk.w, dinv, wk.part_a, wk.part_b, nblk, wk.s, par, it,
                                                thresh);
    SEM_LAUNCH_CHECK("pcg iteration");
    if (it % check_every != 0 && it != opts->maxit) continue;
    SEM_CUDA(cudaMemcpyAsync(&hs, wk.s, sizeof(hs), cudaMemcpyDeviceToHost, st));
    SEM_CUDA(cudaStreamSynchronize(st));
    if (hs.stop_it != 0) return finish(hs.stop_status == 1 ? SEM_OK : SEM_ERR_BREAKDOWN, hs.stop_it, hs.rr);
    if (opts->timeout_s > 0.0) {
      double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > opts->timeout_s) return finish(SEM_ERR_TIMEOUT, it, hs.rr);
    }
  }
  return finish(SEM_ERR_NOT_CONVERGED, opts->maxit, hs.rr);
}

// ---------------------------------------------------------------- no-allocation variant
// The same Jacobi-PCG solve for callers that cannot allocate device memory
// themselves: its workspace is a fixed array in this module's device memory
// (kNoAllocBytes, present on every GPU that loads the library until the
// process exits). The array's device address is looked up once per device
// with cudaGetSymbolAddress, on the first call made with that device current.
namespace {

constexpr size_t kNoAllocBytes = (size_t)64 << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_pcg_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
// per device: the array's address and the context it was looked up in (a
// device reset replaces the context, and the module is loaded anew at
// another address, so the address is looked up again)
void *g_scratch_ptr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);

// the driver's cuCtxGetCurrent, reached through the runtime (no link to libcuda)
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  return fn;
}

int scratch_address(int device, void **out) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (device < 0 || device >= kMaxDevices) return sem_fail(SEM_ERR_INVALID_ARG, "sem_pcg_solve_noalloc: device index out of range");
  CtxGetCurrentFn getctx = ctx_get_current();
  CUcontext ctx = nullptr;
  if (getctx && getctx(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  // look up once per device and context: on the first call, after a device
  // reset, or whenever the current context cannot be identified
  if (!g_scratch_ptr[device] || ctx == nullptr || ctx != g_scratch_ctx[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pcg_scratch);
    if (e != cudaSuccess) return sem_cuda_fail(e, "sem_pcg_solve_noalloc: cudaGetSymbolAddress");
    if (getctx && getctx(&ctx) != CUDA_SUCCESS) ctx = nullptr;  // the lookup makes the context current
    g_scratch_ptr[device] = p;
    g_scratch_ctx[device] = ctx;
  }
  *out = g_scratch_ptr[device];
  return SEM_OK;
}

}  // namespace

extern "C" size_t sem_pcg_noalloc_capacity(void) { return kNoAllocBytes; }

extern "C" int sem_pcg_solve_noalloc(const sem_mesh *m, double h1, double h2, const double *b_g, double *x_g,
                                     const sem_solver_opts *opts, sem_solve_stats *stats, void *stream) {
  if (int rc = check_mesh(m, "sem_pcg_solve_noalloc")) return rc;
  int dev = -1;
  SEM_CUDA(cudaGetDevice(&dev));
  if (dev != m->device)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_pcg_solve_noalloc: the mesh's device must be the current device");
  const size_t need = pcg_layout(m, nullptr, nullptr);
  if (need > kNoAllocBytes) {
    char buf[200];
    snprintf(buf, sizeof(buf),
             "sem_pcg_solve_noalloc: mesh needs %zu bytes of workspace, more than the fixed %zu "
             "(about %zu unique nodes at most); use sem_pcg_solve with caller-provided workspace",
             need, kNoAllocBytes, kNoAllocBytes / (4 * sizeof(double)));
    return sem_fail(SEM_ERR_INVALID_ARG, buf);
  }
  void *ws = nullptr;
  if (int rc = scratch_address(dev, &ws)) return rc;
  return sem_pcg_solve(m, h1, h2, b_g, x_g, opts, ws, stats, stream);
}
