// Element-local field kernels shared by the time-step and adjoint code
// (binary64): inverse Jacobian, physical gradients, advection, weak
// divergence, gathers and small vector operations. Included by one or more
// translation units; each gets its own copy (anonymous namespace).
#pragma once

#include "sem_internal.h"

namespace {

__global__ void k_inv_jacobian(int n, int64_t E, const double *__restrict__ D, const double *__restrict__ X,
                               const double *__restrict__ Y, const double *__restrict__ Z, double *__restrict__ R) {
  const int n3 = n * n * n;
  const int64_t nL = E * n3;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = l / n3;
    const int q = (int)(l - e * n3);
    const int i = q % n, j = (q / n) % n, k = q / (n * n);
    const int64_t base = e * n3;
    const double *xc[3] = {X + base, Y + base, Z + base};
    double J[3][3];
    for (int c = 0; c < 3; ++c) {
      double a = 0, b = 0, d = 0;
      for (int m = 0; m < n; ++m) {
        a = fma(D[i * n + m], xc[c][m + n * (j + n * k)], a);
        b = fma(D[j * n + m], xc[c][i + n * (m + n * k)], b);
        d = fma(D[k * n + m], xc[c][i + n * (j + n * m)], d);
      }
      J[c][0] = a;
      J[c][1] = b;
      J[c][2] = d;
    }
    const double C00 = J[1][1] * J[2][2] - J[1][2] * J[2][1], C01 = J[1][2] * J[2][0] - J[1][0] * J[2][2],
                 C02 = J[1][0] * J[2][1] - J[1][1] * J[2][0], C10 = J[0][2] * J[2][1] - J[0][1] * J[2][2],
                 C11 = J[0][0] * J[2][2] - J[0][2] * J[2][0], C12 = J[0][1] * J[2][0] - J[0][0] * J[2][1],
                 C20 = J[0][1] * J[1][2] - J[0][2] * J[1][1], C21 = J[0][2] * J[1][0] - J[0][0] * J[1][2],
                 C22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double inv = 1.0 / (J[0][0] * C00 + J[0][1] * C01 + J[0][2] * C02);
    const double Rm[9] = {C00 * inv, C10 * inv, C20 * inv, C01 * inv, C11 * inv,
                          C21 * inv, C02 * inv, C12 * inv, C22 * inv};  // [a][c]
    for (int t = 0; t < 9; ++t) R[(9 * e + t) * n3 + q] = Rm[t];
  }
}

__global__ void k_grad(int n, int64_t E, const double *__restrict__ D, const double *__restrict__ R,
                       const double *__restrict__ f, double *__restrict__ gx, double *__restrict__ gy,
                       double *__restrict__ gz) {
  const int n3 = n * n * n;
  const int64_t nL = E * n3;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = l / n3;
    const int q = (int)(l - e * n3);
    const int i = q % n, j = (q / n) % n, k = q / (n * n);
    const double *fe = f + e * n3;
    double dr = 0, ds = 0, dt = 0;
    for (int m = 0; m < n; ++m) {
      dr = fma(D[i * n + m], fe[m + n * (j + n * k)], dr);
      ds = fma(D[j * n + m], fe[i + n * (m + n * k)], ds);
      dt = fma(D[k * n + m], fe[i + n * (j + n * m)], dt);
    }
    const double *Re = R + 9 * e * n3 + q;
    gx[l] = Re[0 * n3] * dr + Re[3 * n3] * ds + Re[6 * n3] * dt;
    gy[l] = Re[1 * n3] * dr + Re[4 * n3] * ds + Re[7 * n3] * dt;
    gz[l] = Re[2 * n3] * dr + Re[5 * n3] * ds + Re[8 * n3] * dt;
  }
}

__global__ void k_neg_adv(int64_t nL, const double *__restrict__ u0, const double *__restrict__ u1,
                          const double *__restrict__ u2, const double *__restrict__ g0, const double *__restrict__ g1,
                          const double *__restrict__ g2, const double *__restrict__ add, double *__restrict__ out) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    double v = -(u0[l] * g0[l] + u1[l] * g1[l] + u2[l] * g2[l]);
    if (add) v += add[l];
    out[l] = v;
  }
}

__global__ void k_weak_div_v(int n, int64_t E, const double *__restrict__ R, const double *__restrict__ B,
                             const double *__restrict__ f0, const double *__restrict__ f1, const double *__restrict__ f2,
                             double *__restrict__ v0, double *__restrict__ v1, double *__restrict__ v2) {
  const int n3 = n * n * n;
  const int64_t nL = E * n3;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = l / n3;
    const int q = (int)(l - e * n3);
    const double *Re = R + 9 * e * n3 + q;
    const double fb0 = f0[l], fb1 = f1[l], fb2 = f2[l], bw = B[l];
    v0[l] = bw * (Re[0 * n3] * fb0 + Re[1 * n3] * fb1 + Re[2 * n3] * fb2);
    v1[l] = bw * (Re[3 * n3] * fb0 + Re[4 * n3] * fb1 + Re[5 * n3] * fb2);
    v2[l] = bw * (Re[6 * n3] * fb0 + Re[7 * n3] * fb1 + Re[8 * n3] * fb2);
  }
}

__global__ void k_dt_sum(int n, int64_t E, const double *__restrict__ D, const double *__restrict__ v0,
                         const double *__restrict__ v1, const double *__restrict__ v2, double *__restrict__ out) {
  const int n3 = n * n * n;
  const int64_t nL = E * n3;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = l / n3;
    const int q = (int)(l - e * n3);
    const int i = q % n, j = (q / n) % n, k = q / (n * n);
    const int64_t base = e * n3;
    double s = 0.0;
    for (int m = 0; m < n; ++m) {
      s = fma(D[m * n + i], v0[base + m + n * (j + n * k)], s);
      s = fma(D[m * n + j], v1[base + i + n * (m + n * k)], s);
      s = fma(D[m * n + k], v2[base + i + n * (j + n * m)], s);
    }
    out[l] = s;
  }
}

__global__ void k_gather_m(int64_t nU, const int32_t *__restrict__ off, const int32_t *__restrict__ perm,
                           const uint8_t *__restrict__ mask, const double *__restrict__ vL, double *__restrict__ vg) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nU; g += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int32_t t = off[g]; t < off[g + 1]; ++t) s += vL[perm[t]];
    vg[g] = (mask && !mask[g]) ? 0.0 : s;
  }
}

__global__ void k_axpbypcz(int64_t n, double a, const double *x, double b, const double *y2, double c,
                           const double *z, double *y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    double v = a * x[g];
    if (y2) v += b * y2[g];
    if (z) v += c * z[g];
    y[g] = v;
  }
}

__global__ void k_lifting(int64_t nL, double Lz, const int32_t *__restrict__ l2g, const double *__restrict__ Z,
                          double *__restrict__ Tb) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL; l += (int64_t)gridDim.x * blockDim.x)
    Tb[l2g[l]] = 1.0 - Z[l] / Lz;  // every copy writes the same value
}

__global__ void k_add_masked(int64_t nU, const uint8_t *__restrict__ mask, const double *__restrict__ a,
                             double *__restrict__ y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nU; g += (int64_t)gridDim.x * blockDim.x)
    if (mask[g]) y[g] += a[g];
}

__global__ void k_sum_part(int64_t n, const double *__restrict__ x, double *__restrict__ part) {
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

__global__ void k_mean_finish(int np, int64_t n, const double *__restrict__ part, double *__restrict__ mean) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < np; ++b) t += part[b];
    *mean = t / (double)n;
  }
}

__global__ void k_sub_scalar(int64_t n, const double *__restrict__ s, double *__restrict__ x) {
  const double v = *s;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    x[g] -= v;
}


}  // namespace
