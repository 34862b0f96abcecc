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
  if (m->slab) return sem_fail(SEM_ERR_INVALID_ARG, "sem_render_slice: needs the whole box, not a partition's slab mesh");
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

// ---------------------------------------------------------------- 3-D iso-surface scene
// The overview scene: iso-surfaces of the field seen in perspective, the box
// walls behind them. The field is first resampled at the cell centres of an
// R_x x R_y x R_z grid of the undeformed box (each value the SEM polynomial
// there: one CTA per element, the element's nodal values in shared memory,
// the grid points inside it evaluated from per-axis Lagrange tables), then
// each pixel's ray marches through the grid with trilinear interpolation in
// steps of one cell, and the first sign change of v - level (for any level)
// is the hit, placed by linear interpolation between the two samples. Colour:
// the colour map at the level times a depth cue (1 at the nearest box corner,
// 1/2 at the farthest); rays without a hit show the colour map of their last
// sample times 0.35; rays missing the box are white. Resampling and marching
// in binary32.
namespace {

struct AxisTab {
  const int32_t *start;  // grid indices of element k along the axis: [start[k], start[k+1])
  const float *basis;    // [R][NP] Lagrange basis at each grid coordinate
};

__global__ void k_resample(int n, int64_t E, int nelx, int nely, const int32_t *__restrict__ l2g,
                           const double *__restrict__ u, AxisTab ax, AxisTab ay, AxisTab az, int Rx, int Ry,
                           float *__restrict__ vol) {
  __shared__ float ue[SEM_MAXNP * SEM_MAXNP * SEM_MAXNP];
  const int n3 = n * n * n;
  for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
    const int ex = (int)(e % nelx), ey = (int)((e / nelx) % nely), ez = (int)(e / ((int64_t)nelx * nely));
    __syncthreads();
    for (int t = threadIdx.x; t < n3; t += blockDim.x) ue[t] = (float)u[l2g[e * n3 + t]];
    __syncthreads();
    const int a0 = ax.start[ex], na = ax.start[ex + 1] - a0;
    const int b0 = ay.start[ey], nb = ay.start[ey + 1] - b0;
    const int c0 = az.start[ez], nc = az.start[ez + 1] - c0;
    const int total = na * nb * nc;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int a = a0 + t % na, b = b0 + (t / na) % nb, c = c0 + t / (na * nb);
      const float *lx = ax.basis + (size_t)a * n, *ly = ay.basis + (size_t)b * n, *lz = az.basis + (size_t)c * n;
      float v = 0.0f;
      for (int k = 0; k < n; ++k) {
        float vk = 0.0f;
        for (int j = 0; j < n; ++j) {
          float vj = 0.0f;
          for (int i = 0; i < n; ++i) vj = fmaf(lx[i], ue[i + n * (j + n * k)], vj);
          vk = fmaf(ly[j], vj, vk);
        }
        v = fmaf(lz[k], vk, v);
      }
      vol[((size_t)c * Ry + b) * Rx + a] = v;
    }
  }
}

struct Cam {
  float eye[3], fw[3], rt[3], up[3];
  float tanh_, aspect;
  float L[3];
  int R[3];
  float h, tnear, tfar, vmin, inv_range;
  int n_iso;
  float iso[4];
};

__device__ __forceinline__ float trilin(const float *__restrict__ vol, const Cam &c, float px, float py, float pz) {
  const float p[3] = {px, py, pz};
  int i0[3];
  float f[3];
  for (int d = 0; d < 3; ++d) {
    float g = fminf(fmaxf(p[d] * c.R[d] / c.L[d] - 0.5f, 0.0f), (float)(c.R[d] - 1));
    if (c.R[d] > 1) {
      i0[d] = min((int)floorf(g), c.R[d] - 2);
      f[d] = g - (float)i0[d];
    } else {
      i0[d] = 0;
      f[d] = 0.0f;
    }
  }
  const size_t sx = 1, sy = (size_t)c.R[0], sz = (size_t)c.R[0] * c.R[1];
  const float *q = vol + i0[2] * sz + i0[1] * sy + i0[0];
  const size_t ox = c.R[0] > 1 ? sx : 0, oy = c.R[1] > 1 ? sy : 0, oz = c.R[2] > 1 ? sz : 0;
  const float x00 = fmaf(f[0], __ldg(q + ox) - __ldg(q), __ldg(q));
  const float x10 = fmaf(f[0], __ldg(q + oy + ox) - __ldg(q + oy), __ldg(q + oy));
  const float x01 = fmaf(f[0], __ldg(q + oz + ox) - __ldg(q + oz), __ldg(q + oz));
  const float x11 = fmaf(f[0], __ldg(q + oz + oy + ox) - __ldg(q + oz + oy), __ldg(q + oz + oy));
  const float y0 = fmaf(f[1], x10 - x00, x00), y1 = fmaf(f[1], x11 - x01, x01);
  return fmaf(f[2], y1 - y0, y0);
}

__device__ __forceinline__ void cmap(float v, float vmin, float inv_range, float &r, float &g, float &b) {
  const float s = fminf(fmaxf((v - vmin) * inv_range, 0.0f), 1.0f);
  if (s < 0.5f) {
    const float f = 2.0f * s;
    r = 59.0f + f * 162.0f;
    g = 76.0f + f * 145.0f;
    b = 192.0f + f * 29.0f;
  } else {
    const float f = 2.0f * s - 1.0f;
    r = 221.0f - f * 41.0f;
    g = 221.0f - f * 217.0f;
    b = 221.0f - f * 183.0f;
  }
}

__global__ void k_scene(int W, int H, Cam c, const float *__restrict__ vol, float *__restrict__ depth,
                        uchar4 *__restrict__ rgba) {
  const int64_t total = (int64_t)W * H;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int py = (int)(t / W), px = (int)(t - (int64_t)py * W);
    const float sx = (2.0f * (px + 0.5f) / W - 1.0f) * c.tanh_ * c.aspect;
    const float sy = (2.0f * (py + 0.5f) / H - 1.0f) * c.tanh_;
    float dr[3];
    float nrm = 0.0f;
    for (int d = 0; d < 3; ++d) {
      dr[d] = c.fw[d] + sx * c.rt[d] + sy * c.up[d];
      nrm = fmaf(dr[d], dr[d], nrm);
    }
    nrm = 1.0f / sqrtf(nrm);
    float t0 = 0.0f, t1 = INFINITY;
    for (int d = 0; d < 3; ++d) {
      dr[d] *= nrm;
      if (dr[d] != 0.0f) {
        const float ta = (0.0f - c.eye[d]) / dr[d], tb = (c.L[d] - c.eye[d]) / dr[d];
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
      } else if (!(c.eye[d] >= 0.0f && c.eye[d] <= c.L[d])) {
        t1 = -1.0f;
      }
    }
    if (t1 < t0) {
      depth[t] = -1.0f;
      rgba[t] = make_uchar4(255, 255, 255, 255);
      continue;
    }
    const int S = (int)floorf((t1 - t0) / c.h);
    float prev = trilin(vol, c, c.eye[0] + t0 * dr[0], c.eye[1] + t0 * dr[1], c.eye[2] + t0 * dr[2]);
    float th = -1.0f, lv = 0.0f;
    for (int s = 1; s <= S; ++s) {
      const float ts = t0 + s * c.h;
      const float cur = trilin(vol, c, c.eye[0] + ts * dr[0], c.eye[1] + ts * dr[1], c.eye[2] + ts * dr[2]);
      for (int q = 0; q < c.n_iso; ++q) {
        const float a = prev - c.iso[q], b = cur - c.iso[q];
        if ((a >= 0.0f) != (b >= 0.0f)) {
          const float tq = ts - c.h + c.h * a / (a - b);
          if (th < 0.0f || tq < th) {
            th = tq;
            lv = c.iso[q];
          }
        }
      }
      if (th >= 0.0f) break;
      prev = cur;
    }
    float r, g, b, shade;
    if (th >= 0.0f) {
      cmap(lv, c.vmin, c.inv_range, r, g, b);
      shade = fminf(fmaxf(1.0f - (th - c.tnear) / (2.0f * (c.tfar - c.tnear)), 0.5f), 1.0f);
    } else {
      cmap(prev, c.vmin, c.inv_range, r, g, b);
      shade = 0.35f;
    }
    depth[t] = th;
    rgba[t] = make_uchar4((unsigned char)floorf(r * shade + 0.5f), (unsigned char)floorf(g * shade + 0.5f),
                          (unsigned char)floorf(b * shade + 0.5f), 255);
  }
}

}  // namespace

extern "C" int sem_render_scene(const sem_mesh *m, const double *u_g, const sem_scene_desc *d, float *volume,
                                float *depth, uint8_t *rgba, void *stream) {
  SemRange nvtx_range("sem_render_scene");
  if (!m || !u_g || !d || !volume || !depth || !rgba) return sem_fail(SEM_ERR_INVALID_ARG, "sem_render_scene: NULL argument");
  if (m->slab) return sem_fail(SEM_ERR_INVALID_ARG, "sem_render_scene: needs the whole box, not a partition's slab mesh");
  if (d->width < 1 || d->height < 1 || d->width > 16384 || d->height > 16384)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_render_scene: width and height must be in [1, 16384]");
  for (int q = 0; q < 3; ++q)
    if (d->grid[q] < 1 || d->grid[q] > 2048) return sem_fail(SEM_ERR_INVALID_ARG, "sem_render_scene: grid must be in [1, 2048]");
  if (!(d->fov_deg > 0.0 && d->fov_deg < 179.0) || !(d->vmax > d->vmin) || d->n_iso < 1 || d->n_iso > 4)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_render_scene: need 0 < fov < 179, vmax > vmin and 1..4 levels");
  double fw[3], rt[3], uu[3];
  for (int q = 0; q < 3; ++q) fw[q] = d->target[q] - d->eye[q];
  auto norm3 = [](double *v) {
    const double s = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(s > 0.0)) return false;
    for (int q = 0; q < 3; ++q) v[q] /= s;
    return true;
  };
  if (!norm3(fw)) return sem_fail(SEM_ERR_INVALID_ARG, "sem_render_scene: eye and target coincide");
  rt[0] = fw[1] * d->up[2] - fw[2] * d->up[1];
  rt[1] = fw[2] * d->up[0] - fw[0] * d->up[2];
  rt[2] = fw[0] * d->up[1] - fw[1] * d->up[0];
  if (!norm3(rt)) return sem_fail(SEM_ERR_INVALID_ARG, "sem_render_scene: up is parallel to the view direction");
  uu[0] = rt[1] * fw[2] - rt[2] * fw[1];
  uu[1] = rt[2] * fw[0] - rt[0] * fw[2];
  uu[2] = rt[0] * fw[1] - rt[1] * fw[0];
  cudaStream_t st = as_stream(stream);
  const int n = m->n;
  // per-axis tables: element of each grid coordinate, its basis values, element ranges
  std::vector<int32_t> starts[3];
  std::vector<float> bases[3];
  std::vector<double> basis(n);
  for (int ax = 0; ax < 3; ++ax) {
    std::vector<double> xk;
    interfaces(m, ax, xk);
    const int R = d->grid[ax];
    std::vector<int32_t> el(R);
    bases[ax].resize((size_t)R * n);
    for (int i = 0; i < R; ++i) {
      el[i] = locate_basis(m, xk, (i + 0.5) * m->L[ax] / R, basis.data());
      for (int q = 0; q < n; ++q) bases[ax][(size_t)i * n + q] = (float)basis[q];
    }
    starts[ax].assign(m->nel[ax] + 1, 0);
    for (int k = 0; k <= m->nel[ax]; ++k)
      starts[ax][k] = (int32_t)(std::lower_bound(el.begin(), el.end(), k) - el.begin());
  }
  size_t bytes = 0;
  for (int ax = 0; ax < 3; ++ax) bytes += sizeof(int32_t) * starts[ax].size() + sizeof(float) * bases[ax].size() + 16;
  char *buf = nullptr;
  if (cudaMalloc((void **)&buf, bytes + 64) != cudaSuccess) return sem_fail(SEM_ERR_NOMEM, "sem_render_scene: cudaMalloc(tables)");
  AxisTab tab[3];
  size_t off = 0;
  cudaError_t e = cudaSuccess;
  for (int ax = 0; ax < 3 && e == cudaSuccess; ++ax) {
    float *b = reinterpret_cast<float *>(buf + off);
    off += ((sizeof(float) * bases[ax].size() + 15) / 16) * 16;
    int32_t *s = reinterpret_cast<int32_t *>(buf + off);
    off += ((sizeof(int32_t) * starts[ax].size() + 15) / 16) * 16;
    e = cudaMemcpyAsync(b, bases[ax].data(), sizeof(float) * bases[ax].size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s, starts[ax].data(), sizeof(int32_t) * starts[ax].size(), cudaMemcpyHostToDevice, st);
    tab[ax].start = s;
    tab[ax].basis = b;
  }
  Cam c;
  for (int q = 0; q < 3; ++q) {
    c.eye[q] = (float)d->eye[q];
    c.fw[q] = (float)fw[q];
    c.rt[q] = (float)rt[q];
    c.up[q] = (float)uu[q];
    c.L[q] = (float)m->L[q];
    c.R[q] = d->grid[q];
  }
  c.tanh_ = (float)tan(d->fov_deg * M_PI / 360.0);
  c.aspect = (float)d->width / (float)d->height;
  c.h = (float)std::min({m->L[0] / d->grid[0], m->L[1] / d->grid[1], m->L[2] / d->grid[2]});
  double tn = INFINITY, tf = 0.0;
  for (int q = 0; q < 8; ++q) {
    const double p[3] = {(q & 1) ? m->L[0] : 0.0, (q & 2) ? m->L[1] : 0.0, (q & 4) ? m->L[2] : 0.0};
    const double dd = sqrt((p[0] - d->eye[0]) * (p[0] - d->eye[0]) + (p[1] - d->eye[1]) * (p[1] - d->eye[1]) +
                           (p[2] - d->eye[2]) * (p[2] - d->eye[2]));
    tn = std::min(tn, dd);
    tf = std::max(tf, dd);
  }
  c.tnear = (float)tn;
  c.tfar = (float)std::max(tf, tn * (1.0 + 1e-6) + 1e-30);
  c.vmin = (float)d->vmin;
  c.inv_range = (float)(1.0 / (d->vmax - d->vmin));
  c.n_iso = d->n_iso;
  for (int q = 0; q < 4; ++q) c.iso[q] = q < d->n_iso ? (float)d->iso[q] : 0.0f;
  if (e == cudaSuccess) {
    const unsigned ge = (unsigned)std::max<int64_t>(1, std::min<int64_t>(m->E, 152 * 16));
    k_resample<<<ge, 128, 0, st>>>(n, m->E, m->nel[0], m->nel[1], m->l2g, u_g, tab[0], tab[1], tab[2], d->grid[0],
                                   d->grid[1], volume);
    const int64_t np = (int64_t)d->width * d->height;
    k_scene<<<grid_for(np, 256), 256, 0, st>>>(d->width, d->height, c, volume, depth,
                                               reinterpret_cast<uchar4 *>(rgba));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return sem_cuda_fail(e, "sem_render_scene");
  return SEM_OK;
}
