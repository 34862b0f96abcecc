// In-situ slice rendering of a spectral-element field into a device image
// (the paper's in-situ scenes, Sec. 5.3 and the figures of Sec. 4.5:
// temperature slices through the plate boundary layers and vertical slices,
// with iso-levels, rendered from data that never leaves the GPU).
//
// A slice is the plane x_a = c of the undeformed box (on a deformed mesh, the
// plane of the reference lattice). Pixel (px, py) is centred at
// ((px + 1/2) L_first / W, (py + 1/2) L_second / H) in the two other axes
// taken in increasing order; row 0 is the low end. Each coordinate is
// located in its element (interfaces uniform, or tanh-stretched along z) with
// a local coordinate in [-1, 1], and the value is the element's polynomial
//   v = sum_{ijk} u(e; i, j, k) l_i l_j l_k
// with l_m the Lagrange basis on the GLL nodes. Two passes: (1) per element of
// the cut layer, the sum over the normal direction in binary64, rounded to
// binary32 (NP^2 values per element); (2) per pixel, the NP x NP in-plane sum
// in binary32, then the colour map (piecewise-linear cool-warm: blue
// (59, 76, 192), grey (221, 221, 221), red (180, 4, 38)) and contour pixels
// (the sign of v - level changes towards the right or upper neighbour).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "sem_internal.h"

namespace {

__global__ void k_slice_reduce(int n, int axis, int ea_n, int eb_n, int ec, int a, int b, int nelx, int nely,
                               const int32_t *__restrict__ l2g, const double *__restrict__ u,
                               const double *__restrict__ Lc, float *__restrict__ S) {
  const int n2 = n * n, n3 = n2 * n;
  const int64_t total = (int64_t)ea_n * eb_n * n2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t el = t / n2;  // element within the layer: ea + ea_n eb
    const int r = (int)(t - el * n2);
    const int ia = r % n, ib = r / n;
    int ecomp[3], comp[3];
    ecomp[a] = (int)(el % ea_n);
    ecomp[b] = (int)(el / ea_n);
    ecomp[axis] = ec;
    const int64_t e = ecomp[0] + (int64_t)nelx * (ecomp[1] + (int64_t)nely * ecomp[2]);
    comp[a] = ia;
    comp[b] = ib;
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
      comp[axis] = k;
      s = fma(u[l2g[e * n3 + comp[0] + n * comp[1] + n2 * comp[2]]], Lc[k], s);
    }
    S[t] = (float)s;
  }
}

__global__ void k_slice_values(int n, int W, int H, int ea_n, const int32_t *__restrict__ colE,
                               const float *__restrict__ La, const int32_t *__restrict__ rowE,
                               const float *__restrict__ Lb, const float *__restrict__ S, float *__restrict__ v) {
  const int n2 = n * n;
  const int64_t total = (int64_t)W * H;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int py = (int)(t / W), px = (int)(t - (int64_t)py * W);
    const float *Se = S + ((int64_t)rowE[py] * ea_n + colE[px]) * n2;
    const float *la = La + (int64_t)px * n, *lb = Lb + (int64_t)py * n;
    float acc = 0.0f;
    for (int ib = 0; ib < n; ++ib) {
      float row = 0.0f;
      for (int ia = 0; ia < n; ++ia) row = fmaf(Se[ib * n + ia], la[ia], row);
      acc = fmaf(row, lb[ib], acc);
    }
    v[t] = acc;
  }
}

struct Iso {
  int n;
  float lvl[8];
};

__device__ __forceinline__ unsigned char chan(float c) { return (unsigned char)floorf(c + 0.5f); }

__global__ void k_slice_color(int W, int H, float vmin, float inv_range, Iso iso, const float *__restrict__ v,
                              uchar4 *__restrict__ rgba) {
  const int64_t total = (int64_t)W * H;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int py = (int)(t / W), px = (int)(t - (int64_t)py * W);
    const float x = v[t];
    uchar4 c;
    if (isnan(x)) {
      c = make_uchar4(255, 0, 255, 255);
    } else {
      const float s = fminf(fmaxf((x - vmin) * inv_range, 0.0f), 1.0f);
      if (s < 0.5f) {
        const float f = 2.0f * s;
        c = make_uchar4(chan(59.0f + f * 162.0f), chan(76.0f + f * 145.0f), chan(192.0f + f * 29.0f), 255);
      } else {
        const float f = 2.0f * s - 1.0f;
        c = make_uchar4(chan(221.0f - f * 41.0f), chan(221.0f - f * 217.0f), chan(221.0f - f * 183.0f), 255);
      }
    }
    bool line = false;
    const float xr = px + 1 < W ? v[t + 1] : x, xu = py + 1 < H ? v[t + W] : x;
    for (int q = 0; q < iso.n; ++q) {
      const bool s0 = x - iso.lvl[q] >= 0.0f;
      line |= (s0 != (xr - iso.lvl[q] >= 0.0f)) || (s0 != (xu - iso.lvl[q] >= 0.0f));
    }
    rgba[t] = line ? make_uchar4(0, 0, 0, 255) : c;
  }
}

void interfaces(const sem_mesh *m, int axis, std::vector<double> &xk) {
  const int n = m->nel[axis];
  const double L = m->L[axis], s = m->desc.z_stretch;
  xk.resize(n + 1);
  for (int k = 0; k <= n; ++k)
    xk[k] = (axis == 2 && s > 0.0) ? 0.5 * L * (1.0 + tanh(s * (2.0 * k / n - 1.0)) / tanh(s)) : k * L / n;
}

// element index and local coordinate of x, then the Lagrange basis there
int locate_basis(const sem_mesh *m, const std::vector<double> &xk, double x, double *basis) {
  const int n = (int)xk.size() - 1;
  int k = (int)(std::upper_bound(xk.begin(), xk.end(), x) - xk.begin()) - 1;
  k = std::min(std::max(k, 0), n - 1);
  const double s = 2.0 * (x - xk[k]) / (xk[k + 1] - xk[k]) - 1.0;
  for (int mth = 0; mth < m->n; ++mth) {
    double p = 1.0;
    for (int q = 0; q < m->n; ++q)
      if (q != mth) p *= (s - m->xi[q]) / (m->xi[mth] - m->xi[q]);
    basis[mth] = p;
  }
  return k;
}

}  // namespace

extern "C" int sem_render_slice(const sem_mesh *m, const double *u_g, const sem_slice_desc *d, float *values,
                                uint8_t *rgba, void *stream) {
  SemRange nvtx_range("sem_render_slice");
  if (!m || !u_g || !d || !values || !rgba) return sem_fail(SEM_ERR_INVALID_ARG, "sem_render_slice: NULL argument");
  if (d->axis < 0 || d->axis > 2 || !(d->coord >= 0.0) || !(d->coord <= m->L[d->axis]))
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_render_slice: axis must be 0..2 and 0 <= coord <= L[axis]");
  if (d->width < 1 || d->height < 1 || d->width > 32768 || d->height > 32768)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_render_slice: width and height must be in [1, 32768]");
  if (!(d->vmax > d->vmin) || d->n_iso < 0 || d->n_iso > 8)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_render_slice: need vmax > vmin and 0 <= n_iso <= 8");
  cudaStream_t st = as_stream(stream);
  const int n = m->n, axis = d->axis;
  const int a = axis == 0 ? 1 : 0, b = axis == 2 ? 1 : 2;  // in-plane axes, increasing
  const int W = d->width, H = d->height;
  std::vector<double> xa, xb, xc;
  interfaces(m, a, xa);
  interfaces(m, b, xb);
  interfaces(m, axis, xc);
  std::vector<int32_t> colE(W), rowE(H);
  std::vector<float> La((size_t)W * n), Lb((size_t)H * n);
  std::vector<double> basis(n), Lc(n);
  for (int px = 0; px < W; ++px) {
    colE[px] = locate_basis(m, xa, (px + 0.5) * m->L[a] / W, basis.data());
    for (int q = 0; q < n; ++q) La[(size_t)px * n + q] = (float)basis[q];
  }
  for (int py = 0; py < H; ++py) {
    rowE[py] = locate_basis(m, xb, (py + 0.5) * m->L[b] / H, basis.data());
    for (int q = 0; q < n; ++q) Lb[(size_t)py * n + q] = (float)basis[q];
  }
  const int ec = locate_basis(m, xc, d->coord, Lc.data());
  const int ea_n = m->nel[a], eb_n = m->nel[b];
  const size_t nS = (size_t)ea_n * eb_n * n * n;
  // one scratch allocation per call: the per-pixel tables and the layer sums
  const size_t bytes = sizeof(int32_t) * (W + H) + sizeof(float) * ((size_t)(W + H) * n + nS) + sizeof(double) * n;
  char *buf = nullptr;
  if (cudaMalloc((void **)&buf, bytes + 64) != cudaSuccess)
    return sem_fail(SEM_ERR_NOMEM, "sem_render_slice: cudaMalloc(tables)");
  double *dLc = reinterpret_cast<double *>(buf);
  float *dS = reinterpret_cast<float *>(buf + sizeof(double) * n);
  float *dLa = dS + nS, *dLb = dLa + (size_t)W * n;
  int32_t *dcol = reinterpret_cast<int32_t *>(dLb + (size_t)H * n), *drow = dcol + W;
  cudaError_t e = cudaMemcpyAsync(dLc, Lc.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dLa, La.data(), sizeof(float) * La.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dLb, Lb.data(), sizeof(float) * Lb.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dcol, colE.data(), sizeof(int32_t) * W, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(drow, rowE.data(), sizeof(int32_t) * H, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_slice_reduce<<<grid_for((int64_t)nS, 256), 256, 0, st>>>(n, axis, ea_n, eb_n, ec, a, b, m->nel[0], m->nel[1],
                                                               m->l2g, u_g, dLc, dS);
    const int64_t np = (int64_t)W * H;
    k_slice_values<<<grid_for(np, 256), 256, 0, st>>>(n, W, H, ea_n, dcol, dLa, drow, dLb, dS, values);
    Iso iso;
    iso.n = d->n_iso;
    for (int q = 0; q < 8; ++q) iso.lvl[q] = q < d->n_iso ? (float)d->iso[q] : 0.0f;
    k_slice_color<<<grid_for(np, 256), 256, 0, st>>>(W, H, (float)d->vmin, (float)(1.0 / (d->vmax - d->vmin)), iso,
                                                     values, reinterpret_cast<uchar4 *>(rgba));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the tables are freed below
  cudaFree(buf);
  if (e != cudaSuccess) return sem_cuda_fail(e, "sem_render_slice");
  return SEM_OK;
}

extern "C" int sem_write_ppm(const char *path, const uint8_t *rgba_host, int width, int height) {
  if (!path || !rgba_host || width < 1 || height < 1)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_write_ppm: bad argument");
  FILE *f = fopen(path, "wb");
  if (!f) return sem_fail(SEM_ERR_IO, std::string("sem_write_ppm: cannot open ") + path);
  fprintf(f, "P6\n%d %d\n255\n", width, height);
  std::vector<unsigned char> row((size_t)width * 3);
  bool ok = true;
  for (int y = height - 1; y >= 0 && ok; --y) {  // the top of the file is the high end of the image
    for (int x = 0; x < width; ++x)
      for (int c = 0; c < 3; ++c) row[(size_t)x * 3 + c] = rgba_host[((size_t)y * width + x) * 4 + c];
    ok = fwrite(row.data(), 1, row.size(), f) == row.size();
  }
  if (fclose(f) != 0 || !ok) return sem_fail(SEM_ERR_IO, std::string("sem_write_ppm: write failed: ") + path);
  return SEM_OK;
}
