// Smoothing-level operator at N = 7 in bfloat16 on the tensor cores (Sec. 2.2:
// the leading-order work is dense (p+1)x(p+1) tensor contractions, and most
// of the preconditioner runs in reduced precision).
//
// w[g] += h1 (A u)[g] + h2 (B u)[g] through the level's map. Geometric
// factors are bfloat16. D, u and the metric's outputs enter the tensor cores
// as two-part bfloat16 values (x = x_hi + x_lo to 2^-17). Each contraction
// forms the three products hi x hi, D_lo x hi and D_hi x lo, accumulated in
// binary32, so the operator is accurate to about 2^-15 of |D|^T|G||D||u|.
// Rounding u and the metric's outputs to a single bfloat16 instead (2^-8)
// was measured: the smoothing then raised the outer p-multigrid iterations
// from 12 to 21 on the 64^3 Poisson problem and from 5 to 13-15 in the
// Rayleigh-Benard pressure solve.
//
// One warp per element at a time; the element's fields stay in registers
// (inputs arrive through shared memory, see below). Lane (g, q) = (lane / 4,
// lane % 4) owns the 16 points (i, j, k) = (g, 2q + jj, k), jj = 0, 1,
// k = 0..7: for every k-plane the pair (j = 2q, 2q + 1) at row i = g, which
// is both the A-fragment and the accumulator layout of mma m16n8k16, and
// for both of its (i, j) columns the whole k-line. Two k-planes k1, k2 are
// stacked in one mma against a block-diagonal operand:
//   r (contracted over i): A = diag(D, D), B = [U_k1^T; U_k2^T] (the planes
//       transposed by movmatrix);
//   s (contracted over j): A = diag(U_k1, U_k2), B = [D^T; D^T];
// and the accumulator holds the result at the lane's own points (rows 0-7
// plane k1, rows 8-15 plane k2). The t-lines are thread-local: binary32
// multiply-adds with D from constant memory. The metric (wr, ws, wt) =
// G (ur, us, ut) is binary32; wr and ws are split into two bfloat16 parts
// for the transposed r and s contractions (same forms with D^T), which
// accumulate into one fragment, and the transposed t-line is added in
// binary32.
//
// Memory per local point: G 12 B and the map 4 B, read as 16-byte vectors
// from lane-major copies made at set-up, u gathered and w scattered once
// per unique node (binary32): about 21 B, the same as the bfloat16-geometry
// binary32 kernel it replaces at this order. The warps are persistent and
// pipeline two elements each: cp.async brings the next element's u values
// (through the map) and geometry into one shared-memory slot while the
// current element is computed from the other. Each lane copies, and later
// reads, only its own words, so the slots need no barrier.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "sem_internal.h"

namespace {

constexpr int NP = 8, N3 = 512;
constexpr int kWarps = 4;  // elements per CTA

// Lane-major copies, per element e and lane L = 4g + q (the lane's points
// P(k, jj) = g + 8 (2q + jj) + 64 k):
//   G: 12 uint4 per lane; uint4 c = 3a + b holds, for the plane pair
//      (2a, 2a + 1), factors f = 2b, 2b + 1 as bfloat16 pairs (jj = 0, 1):
//      word 2 (f - 2b) + kl = (G_f(P(2a + kl, 0)), G_f(P(2a + kl, 1)));
//      stored [e][c][L] so that each uint4 load of a warp is 512 contiguous bytes;
//   map: 4 int4 per lane, int4 c = (P(2c, 0), P(2c, 1), P(2c + 1, 0), P(2c + 1, 1));
//   B (Helmholtz levels only): 4 float4 per lane, the same order as the map.
__device__ __forceinline__ int lane_point(int lane, int k, int jj) {
  return (lane >> 2) + 8 * (2 * (lane & 3) + jj) + 64 * k;
}

__global__ void k_bf16_pack(int64_t E, const double *__restrict__ G, const int32_t *__restrict__ map,
                            const double *__restrict__ B, uint4 *__restrict__ Gl, int4 *__restrict__ Ml,
                            float4 *__restrict__ Bl) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < E * 32; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t >> 5;
    const int lane = (int)(t & 31);
    const double *Ge = G + e * 6 * N3;
    for (int c = 0; c < 12; ++c) {
      const int a = c / 3, b = c % 3;
      uint32_t wv[4];
      for (int fl = 0; fl < 2; ++fl)
        for (int kl = 0; kl < 2; ++kl) {
          const int f = 2 * b + fl, k = 2 * a + kl;
          const __nv_bfloat16 v0 = __double2bfloat16(Ge[f * N3 + lane_point(lane, k, 0)]);
          const __nv_bfloat16 v1 = __double2bfloat16(Ge[f * N3 + lane_point(lane, k, 1)]);
          wv[2 * fl + kl] = (uint32_t)__bfloat16_as_ushort(v0) | ((uint32_t)__bfloat16_as_ushort(v1) << 16);
        }
      Gl[(e * 12 + c) * 32 + lane] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
    for (int c = 0; c < 4; ++c) {
      const int p00 = lane_point(lane, 2 * c, 0), p01 = lane_point(lane, 2 * c, 1);
      const int p10 = lane_point(lane, 2 * c + 1, 0), p11 = lane_point(lane, 2 * c + 1, 1);
      Ml[(e * 4 + c) * 32 + lane] =
          make_int4(map[e * N3 + p00], map[e * N3 + p01], map[e * N3 + p10], map[e * N3 + p11]);
      if (Bl)
        Bl[(e * 4 + c) * 32 + lane] = make_float4((float)B[e * N3 + p00], (float)B[e * N3 + p01],
                                                  (float)B[e * N3 + p10], (float)B[e * N3 + p11]);  // set-up only
    }
  }
}

// D at N = 7 in binary32 (the t-lines) and its split D = D_hi + D_lo into
// bfloat16 parts (the mma operands), from the host's GLL set-up
__constant__ float c_D8[NP * NP];
std::mutex g_d8_mu;
unsigned g_d8_ready = 0;  // bit per device

int ensure_d8(int device) {
  std::lock_guard<std::mutex> lk(g_d8_mu);
  if (device < 32 && (g_d8_ready >> device) & 1u) return SEM_OK;
  double xi[SEM_MAXNP], rho[SEM_MAXNP], D[SEM_MAXNP * SEM_MAXNP];
  if (int rc = sem_gll_host(NP - 1, xi, rho, D)) return rc;
  float Df[NP * NP];
  for (int t = 0; t < NP * NP; ++t) Df[t] = (float)D[t];
  SEM_CUDA(cudaMemcpyToSymbol(c_D8, Df, sizeof(Df)));
  if (device < 32) g_d8_ready |= 1u << device;
  return SEM_OK;
}

// d = a b + d, m16n8k16, bfloat16 operands, binary32 accumulate. Fragments
// (lane = 4g + q): a0 (row g, cols 2q, 2q+1), a1 (row g+8), a2 (row g, cols
// 2q+8, 2q+9), a3 (row g+8, cols 2q+8, 2q+9); b0 (rows 2q, 2q+1, col g), b1
// (rows 2q+8, 2q+9); d0, d1 (row g, cols 2q, 2q+1), d2, d3 (row g+8). The
// lower column (row) of a pair is the low half of its register.
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// transpose of the 8x8 bfloat16 matrix whose row g, cols 2q, 2q+1 this lane holds
__device__ __forceinline__ uint32_t trans8(uint32_t a) {
  uint32_t d;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;\n" : "=r"(d) : "r"(a));
  return d;
}

// (lo, hi) -> bfloat16 pair, round to nearest even; and back
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}
__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }
__device__ __forceinline__ float bf_half(uint32_t v, int jj) { return jj ? bf_hi(v) : bf_lo(v); }

// bfloat16 parts of d: hi = bf16(d), lo = bf16(d - hi) (d - hi is exact in binary32)
__device__ __forceinline__ void split_bf16(float d, float &hi, float &lo) {
  hi = __bfloat162float(__float2bfloat16_rn(d));
  lo = __bfloat162float(__float2bfloat16_rn(d - hi));
}

// asynchronous global -> shared copies (each lane copies, and later reads, its own words)
__device__ __forceinline__ void cp16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp4(void *dst, const float *src, bool valid) {  // zero-filled when !valid
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Shared memory per warp: two slots, each one element's lane-major geometry
// (12 x 32 uint4) and gathered u values (4 x 32 float4, the map's order).
constexpr int kSlotG = 12 * 32;                       // uint4 per slot
constexpr int kSlotU = 4 * 32;                        // float4 per slot
constexpr int kWarpSmem = 2 * (kSlotG + kSlotU) * 16;  // bytes
constexpr int kSmem = kWarps * kWarpSmem;              // 64 KB per CTA

template <bool HELM>
__global__ void __launch_bounds__(kWarps * 32, 3)
    k_ax_bf16(int64_t E, const uint4 *__restrict__ Gl, const int4 *__restrict__ Ml, const float4 *__restrict__ Bl,
              float h1, float h2, const float *__restrict__ u, float *__restrict__ w, float *__restrict__ wloc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
  // F = (D[g][2q], D[g][2q+1]): A of the forward r-contraction and B of the
  // forward s-contraction; T = (D[2q][g], D[2q+1][g]): the same roles in the
  // transposed contractions. Each as its bfloat16 hi and lo parts.
  uint32_t Fh, Fl, Th, Tl;
  {
    float h0, l0, h1v, l1v;
    split_bf16(c_D8[g * NP + 2 * q], h0, l0);
    split_bf16(c_D8[g * NP + 2 * q + 1], h1v, l1v);
    Fh = pack_bf16(h0, h1v);
    Fl = pack_bf16(l0, l1v);
    split_bf16(c_D8[(2 * q) * NP + g], h0, l0);
    split_bf16(c_D8[(2 * q + 1) * NP + g], h1v, l1v);
    Th = pack_bf16(h0, h1v);
    Tl = pack_bf16(l0, l1v);
  }
  // Persistent warps, each over elements e = w0, w0 + nw, ...: while one
  // element is computed from its slot, the next element's u values (through
  // the map) and geometry are in flight into the other slot.
  extern __shared__ __align__(16) uint4 sm4[];
  uint4 *const wbase = sm4 + warp * (kWarpSmem / 16);  // slot sl: geometry at sl (G + U), then u
  auto slot_g = [&](int sl) { return wbase + sl * (kSlotG + kSlotU); };
  auto prefetch = [&](int64_t en, int sl) {
    float *du = reinterpret_cast<float *>(slot_g(sl) + kSlotG);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int4 mc = __ldg(&Ml[(en * 4 + c) * 32 + lane]);
      float *d = du + 4 * (c * 32 + lane);
      cp4(d, u + (mc.x >= 0 ? mc.x : 0), mc.x >= 0);
      cp4(d + 1, u + (mc.y >= 0 ? mc.y : 0), mc.y >= 0);
      cp4(d + 2, u + (mc.z >= 0 ? mc.z : 0), mc.z >= 0);
      cp4(d + 3, u + (mc.w >= 0 ? mc.w : 0), mc.w >= 0);
    }
#pragma unroll
    for (int c = 0; c < 12; ++c) cp16(slot_g(sl) + c * 32 + lane, Gl + (en * 12 + c) * 32 + lane);
  };
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  int64_t e = (int64_t)blockIdx.x * kWarps + warp;  // warp-uniform
  if (e < E) prefetch(e, 0);
  cp_commit();
  for (int sl = 0; e < E; e += nw, sl ^= 1) {
    if (e + nw < E) prefetch(e + nw, sl ^ 1);
    cp_commit();
    cp_wait_prev();  // this lane's copies of element e have landed
    const uint4 *sg = slot_g(sl);
    const float4 *su = reinterpret_cast<const float4 *>(sg + kSlotG);
    // u at the lane's 16 points as two-part bfloat16 pairs:
    // U[k] + V[k] = (u(g, 2q, k), u(g, 2q+1, k)) to 2^-17
    uint32_t U[NP], V[NP];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 uv = su[c * 32 + lane];
      const float v00 = uv.x, v01 = uv.y, v10 = uv.z, v11 = uv.w;
      U[2 * c] = pack_bf16(v00, v01);
      U[2 * c + 1] = pack_bf16(v10, v11);
      V[2 * c] = pack_bf16(v00 - bf_lo(U[2 * c]), v01 - bf_hi(U[2 * c]));
      V[2 * c + 1] = pack_bf16(v10 - bf_lo(U[2 * c + 1]), v11 - bf_hi(U[2 * c + 1]));
    }
    // acc: the lane's 16 outputs, (A u)(g, 2q + jj, k) = acc[k][jj]
    float acc[NP][2];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k][0] = acc[k][1] = 0.0f;
#pragma unroll
    for (int a = 0; a < NP / 2; ++a) {
      const int k1 = 2 * a, k2 = 2 * a + 1;
      // forward t-lines at the two planes (binary32)
      float ut[2][2];
#pragma unroll
      for (int kl = 0; kl < 2; ++kl)
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          float sum = 0.0f;
#pragma unroll
          for (int m = 0; m < NP; ++m)
            sum = fmaf(c_D8[(k1 + kl) * NP + m], bf_half(U[m], jj) + bf_half(V[m], jj), sum);
          ut[kl][jj] = sum;
        }
      // forward r and s of the plane pair; d[2 kl + jj] is the point (k1 + kl, jj)
      float cr[4] = {0.0f, 0.0f, 0.0f, 0.0f}, cs[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      // three products of the two-part operands: hi x hi, lo(D) x hi, hi(D) x lo
      const uint32_t b0 = trans8(U[k1]), b1 = trans8(U[k2]);
      const uint32_t c0 = trans8(V[k1]), c1 = trans8(V[k2]);
      mma_bf16(cr, Fh, 0u, 0u, Fh, b0, b1);
      mma_bf16(cr, Fl, 0u, 0u, Fl, b0, b1);
      mma_bf16(cr, Fh, 0u, 0u, Fh, c0, c1);
      mma_bf16(cs, U[k1], 0u, 0u, U[k2], Fh, Fh);
      mma_bf16(cs, U[k1], 0u, 0u, U[k2], Fl, Fl);
      mma_bf16(cs, V[k1], 0u, 0u, V[k2], Fh, Fh);
      // metric: factor f of point (kl, jj) is half jj of word 2 (f % 2) + kl of G[f / 2]
      const uint4 G0 = sg[(3 * a) * 32 + lane];
      const uint4 G1 = sg[(3 * a + 1) * 32 + lane];
      const uint4 G2 = sg[(3 * a + 2) * 32 + lane];
      float wr[4], ws[4], wt[4];
#pragma unroll
      for (int idx = 0; idx < 4; ++idx) {
        const int kl = idx >> 1, jj = idx & 1;
        const float g00 = bf_half(kl ? G0.y : G0.x, jj), g01 = bf_half(kl ? G0.w : G0.z, jj);
        const float g02 = bf_half(kl ? G1.y : G1.x, jj), g11 = bf_half(kl ? G1.w : G1.z, jj);
        const float g12 = bf_half(kl ? G2.y : G2.x, jj), g22 = bf_half(kl ? G2.w : G2.z, jj);
        const float ur = cr[idx], us = cs[idx], uu = ut[kl][jj];
        wr[idx] = fmaf(g00, ur, fmaf(g01, us, g02 * uu));
        ws[idx] = fmaf(g01, ur, fmaf(g11, us, g12 * uu));
        wt[idx] = fmaf(g02, ur, fmaf(g12, us, g22 * uu));
      }
      // transposed t-lines: planes k1, k2 contribute D[k1][k] wt(k1) + D[k2][k] wt(k2) to every plane k
#pragma unroll
      for (int k = 0; k < NP; ++k)
#pragma unroll
        for (int jj = 0; jj < 2; ++jj)
          acc[k][jj] = fmaf(c_D8[k1 * NP + k], wt[jj], fmaf(c_D8[k2 * NP + k], wt[2 + jj], acc[k][jj]));
      // transposed r and s into one fragment
      const uint32_t WR1 = pack_bf16(wr[0], wr[1]), WR2 = pack_bf16(wr[2], wr[3]);
      const uint32_t WS1 = pack_bf16(ws[0], ws[1]), WS2 = pack_bf16(ws[2], ws[3]);
      const uint32_t XR1 = pack_bf16(wr[0] - bf_lo(WR1), wr[1] - bf_hi(WR1));
      const uint32_t XR2 = pack_bf16(wr[2] - bf_lo(WR2), wr[3] - bf_hi(WR2));
      const uint32_t XS1 = pack_bf16(ws[0] - bf_lo(WS1), ws[1] - bf_hi(WS1));
      const uint32_t XS2 = pack_bf16(ws[2] - bf_lo(WS2), ws[3] - bf_hi(WS2));
      float co[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      const uint32_t t0 = trans8(WR1), t1 = trans8(WR2), x0 = trans8(XR1), x1 = trans8(XR2);
      mma_bf16(co, Th, 0u, 0u, Th, t0, t1);
      mma_bf16(co, Tl, 0u, 0u, Tl, t0, t1);
      mma_bf16(co, Th, 0u, 0u, Th, x0, x1);
      mma_bf16(co, WS1, 0u, 0u, WS2, Th, Th);
      mma_bf16(co, WS1, 0u, 0u, WS2, Tl, Tl);
      mma_bf16(co, XS1, 0u, 0u, XS2, Th, Th);
      acc[k1][0] += co[0];
      acc[k1][1] += co[1];
      acc[k2][0] += co[2];
      acc[k2][1] += co[3];
    }
    // h1 A u (+ h2 B u) to the lane's points
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int4 mc = __ldg(&Ml[(e * 4 + c) * 32 + lane]);  // again (cached): not held across the element
      const int gi[4] = {mc.x, mc.y, mc.z, mc.w};
      float bv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (HELM) {
        const float4 b4 = Bl[(e * 4 + c) * 32 + lane];
        bv[0] = b4.x;
        bv[1] = b4.y;
        bv[2] = b4.z;
        bv[3] = b4.w;
      }
#pragma unroll
      for (int idx = 0; idx < 4; ++idx) {
        const int k = 2 * c + (idx >> 1), jj = idx & 1;
        float val = h1 * acc[k][jj];
        if (HELM) val = fmaf(h2 * bv[idx], bf_half(U[k], jj) + bf_half(V[k], jj), val);
        if (wloc) wloc[e * N3 + lane_point(lane, k, jj)] = gi[idx] >= 0 ? val : 0.0f;
        else if (gi[idx] >= 0) atomicAdd(&w[gi[idx]], val);
      }
    }
  }
  cp_wait_all();  // no copy is left in flight when the warp exits
}

}  // namespace

// bytes of the lane-major copies for a mesh at N = 7
size_t sem_bf16_layout_bytes(const sem_mesh *m, int which) {
  const size_t E = (size_t)m->E;
  if (which == 0) return E * 12 * 32 * sizeof(uint4);  // G
  return E * 4 * 32 * sizeof(int4);                    // map (and B, which is as large)
}

// Fill the lane-major copies of the level's geometry, map and (Helmholtz
// levels) mass from the mesh (binary64 G and B). Gl, Ml: device buffers of
// sem_bf16_layout_bytes(m, 0) and (m, 1) bytes; Bl: NULL or (m, 1) bytes.
int sem_bf16_pack(const sem_mesh *m, const int32_t *map, void *Gl, void *Ml, void *Bl, cudaStream_t st) {
  if (m->n != NP) return sem_fail(SEM_ERR_INVALID_ARG, "bfloat16 tensor-core operator: N = 7 only");
  k_bf16_pack<<<grid_for(m->E * 32, 256), 256, 0, st>>>(m->E, m->G, map, m->B, (uint4 *)Gl, (int4 *)Ml,
                                                         (float4 *)Bl);
  SEM_LAUNCH_CHECK("k_bf16_pack");
  return SEM_OK;
}

// w += h1 A u + h2 B u (binary32 vectors, bfloat16 arithmetic with binary32
// accumulation); wloc: the deterministic mode's E-vector (then w untouched
// here and summed by the caller), else NULL.
int sem_launch_ax_bf16(const sem_mesh *m, const void *Gl, const void *Ml, const void *Bl, float h1, float h2,
                       const float *u, float *w, float *wloc, cudaStream_t st) {
  if (m->n != NP) return sem_fail(SEM_ERR_INVALID_ARG, "bfloat16 tensor-core operator: N = 7 only");
  if (h2 != 0.0f && !Bl) return sem_fail(SEM_ERR_INVALID_ARG, "bfloat16 tensor-core operator: no mass copy");
  if (int rc = ensure_d8(m->device)) return rc;
  auto kern = h2 != 0.0f ? k_ax_bf16<true> : k_ax_bf16<false>;
  SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  // persistent: the CTAs that fit on the GPU at once, at most one warp per element
  int per_sm = 0, nsm = 0;
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarps * 32, kSmem));
  SEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
  const int64_t need = (m->E + kWarps - 1) / kWarps;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)std::max(per_sm, 1) * nsm));
  kern<<<grid, kWarps * 32, kSmem, st>>>(m->E, (const uint4 *)Gl, (const int4 *)Ml,
                                         h2 != 0.0f ? (const float4 *)Bl : nullptr, h1, h2, u, w, wloc);
  SEM_LAUNCH_CHECK("k_ax_bf16");
  return SEM_OK;
}
