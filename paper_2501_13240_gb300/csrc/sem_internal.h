// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "sem.h"

// NVTX range over an entry point (visible in Nsight timelines; a no-op when
// no tool is attached)
struct SemRange {
  explicit SemRange(const char *name) { nvtxRangePushA(name); }
  ~SemRange() { nvtxRangePop(); }
  SemRange(const SemRange &) = delete;
  SemRange &operator=(const SemRange &) = delete;
};

#define SEM_MAXN 10
#define SEM_MAXNP (SEM_MAXN + 1)

struct sem_mesh {
  sem_box_desc desc;  // the description the mesh was built from
  int nel[3];
  int N;
  int n;          // N + 1
  int n3;         // (N + 1)^3
  int64_t E;
  int64_t n_local;
  int64_t n_unique;
  int periodic[3];
  int dirichlet[6];
  double L[3];
  double detJ_min;
  double xi[SEM_MAXNP], rho[SEM_MAXNP], D[SEM_MAXNP * SEM_MAXNP];
  // device arrays (owned)
  double *X = nullptr, *Y = nullptr, *Z = nullptr;
  double *G = nullptr;      // [E][6][n3]
  float2 *Gdf = nullptr;    // [E][6][n3] double-float split of G (hi, lo)
  double *B = nullptr;      // [E][n3]
  float2 *Bdf = nullptr;    // [E][n3] double-float split of B
  int32_t *l2g = nullptr;   // [n_local]
  int32_t *l2gm = nullptr;  // [n_local] l2g, or -1 on Dirichlet nodes
  uint8_t *mask = nullptr;  // [n_unique]
  double *mult = nullptr;   // [n_unique]
  int32_t *gs_off = nullptr;   // [n_unique + 1]
  int32_t *gs_perm = nullptr;  // [n_local]
  double *dD = nullptr;     // device copy of D (n*n)
  int device = 0;
  // deterministic assembly: when set, assembled operators write element
  // results here (n_local doubles, or floats for binary32 levels) and sum the
  // copies of each unique node in ascending copy order instead of with atomics
  void *det_w = nullptr;
  // N = 7 double-float operator: 1-D contractions on the tensor pipe
  // (sem_ax_tc.cu) when set (the default), else on the binary32 pipe
  int use_tc = 0;  // N = 7 double-float route: 0 binary32 pipe, 1 tensor cores, 2 tensor cores register-resident
  void *Gt = nullptr, *Mt = nullptr;  // lane-major geometry and masked map of the register-resident route
  // a slab of element planes of a box (a partition's share, sem_part): its
  // own unique numbering, no periodic wrap in z; first plane slab_p0
  int slab = 0;
  int slab_p0 = 0;
  // N = 1 only: element stiffness matrices (upper triangle, [36][E]) in
  // binary64 and double-float
  double *K1 = nullptr;
  float2 *K1df = nullptr;
};

int sem_mesh_create_slab(const sem_box_desc *d, int p0, int p1, void *stream, sem_mesh **out);

// thread-local error reporting
int sem_fail(int code, const std::string &msg);
int sem_cuda_fail(cudaError_t e, const char *what);
#define SEM_CUDA(call)                                              \
  do {                                                              \
    cudaError_t _e = (call);                                        \
    if (_e != cudaSuccess) return sem_cuda_fail(_e, #call);         \
  } while (0)
#define SEM_LAUNCH_CHECK(what)                                      \
  do {                                                              \
    cudaError_t _e = cudaGetLastError();                            \
    if (_e != cudaSuccess) return sem_cuda_fail(_e, what);          \
  } while (0)

static inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// host-side GLL (long double Newton), shared by the set-up code
int sem_gll_host(int N, double *xi, double *rho, double *D);

// kernels launched from other translation units
int sem_launch_ax_local(const sem_mesh *m, double h1, double h2, const double *u, double *w,
                        int precision, cudaStream_t st);
// map: local-to-unique map to gather/scatter through (nullptr: the masked
// map l2gm; m->l2g for the unmasked operator). skip: a device flag read by the
// kernel when it starts; non-zero makes the launch a no-op (w and the p.w
// partials untouched) so a solve can queue iterations past its stopping point
int sem_launch_ax_assembled(const sem_mesh *m, double h1, double h2, const double *u_g, double *w_g,
                            double *pw_partial, int precision, cudaStream_t st, const int32_t *map = nullptr,
                            const int *skip = nullptr);
int sem_ax_assembled_blocks(const sem_mesh *m, int precision);
// the assembled operator over a device list of elements only: w_g +=
// M Q_e^T A_e Q_e M u_g for the listed e (atomic assembly, no p.w partials)
int sem_launch_ax_assembled_list(const sem_mesh *m, double h1, double h2, const double *u_g, double *w_g,
                                 int precision, cudaStream_t st, const int32_t *elist, int64_t nlist);
int sem_launch_ax_df64_list(const sem_mesh *m, double h1, double h2, const double *u, double *w, cudaStream_t st,
                            const int32_t *elist, int64_t nlist);
// bfloat16 tensor-core operator of the N = 7 smoothing level (sem_ax_bf16.cu):
// sizes of its lane-major copies (which = 0: geometry; 1: map, and mass),
// their set-up, and the launch (w += h1 A u + h2 B u, binary32 vectors)
size_t sem_bf16_layout_bytes(const sem_mesh *m, int which);
int sem_bf16_pack(const sem_mesh *m, const int32_t *map, void *Gl, void *Ml, void *Bl, cudaStream_t st);
int sem_launch_ax_bf16(const sem_mesh *m, const void *Gl, const void *Ml, const void *Bl, float h1, float h2,
                       const float *u, float *w, float *wloc, cudaStream_t st);
// number of p.w partial sums the double-float assembled operator writes (both
// routes at N = 7: one per warp of the sum-factorised kernel's CTAs)
int sem_df64_pw_count(const sem_mesh *m);
int sem_launch_ax_df64(const sem_mesh *m, double h1, double h2, const double *u, double *w, double *pw_partial,
                       bool assembled, cudaStream_t st, const int32_t *map, const int *skip = nullptr);
// fill the register-resident route's lane-major copies (N = 7)
int sem_tcr_prepare(sem_mesh *m, cudaStream_t st);
// the register-resident route: Poisson operator (h1 = 1, h2 = 0), masked map
int sem_launch_ax_tcr(const sem_mesh *m, const double *u, double *w, double *pw_partial, bool assembled,
                      cudaStream_t st, const int *skip);
int sem_launch_ax_tc(const sem_mesh *m, double h1, double h2, const double *u, double *w, double *pw_partial,
                     bool assembled, cudaStream_t st, const int32_t *map, const int *skip,
                     const int32_t *elist = nullptr, int64_t nlist = 0);
int sem_launch_gs(const sem_mesh *m, double *v, int apply_mask, cudaStream_t st);
int sem_launch_gather(const sem_mesh *m, const double *vL, double *vg, cudaStream_t st);
int sem_launch_scatter(const sem_mesh *m, const double *vg, double *vL, cudaStream_t st);
// w[g] += sum over the copies of g (ascending) of wL; the deterministic
// replacement of atomic assembly
int sem_launch_gather_add(const sem_mesh *m, const double *wL, double *w, cudaStream_t st);
// N = 1 meshes: element matrices (set-up) and the assembled operator from them
int sem_n1_prepare(sem_mesh *m, cudaStream_t st);
int sem_launch_ax_n1(const sem_mesh *m, double h1, double h2, const double *u_g, double *w_g, double *pw_partial,
                     int precision, cudaStream_t st, const int32_t *map, const int *skip = nullptr);
// Jacobi-PCG on an N = 1 mesh in one cooperative launch (the p-multigrid
// coarsest level); synchronises the stream
size_t sem_pcg_n1_workspace_bytes(const sem_mesh *m);
int sem_pcg_n1_persistent(const sem_mesh *m, double h1, double h2, const double *b, double *x, const double *dinv,
                          const int32_t *map, double tol, int maxit, void *work, int *iters, double *rel,
                          cudaStream_t st);
// polls (of about 0.1 us) after which a grid-barrier wait of a cooperative
// kernel gives up and the kernel ends with an error flag (sem_set_grid_wait_limit)
unsigned sem_grid_wait_limit();
int sem_launch_gather_add_f(const sem_mesh *m, const float *wL, float *w, cudaStream_t st);
// binary64-accurate element-local field operators in double-float
// arithmetic; Rdf = the inverse Jacobian dr_a/dx_c split to (hi, lo),
// [E][9][n3] with factor 3a + c. grad: g_c = sum_a dr_a/dx_c D_a f (E-vectors
// in and out); wdiv: out = sum_a D_a^T (B sum_c dr_a/dx_c f_c)
int sem_launch_grad_df64(const sem_mesh *m, const float2 *Rdf, const double *f, double *g0, double *g1, double *g2,
                         cudaStream_t st);
int sem_launch_wdiv_df64(const sem_mesh *m, const float2 *Rdf, const double *f0, const double *f1, const double *f2,
                         double *out, cudaStream_t st);
int sem_launch_split_df64(const double *x, float2 *y, int64_t n, cudaStream_t st);
int sem_launch_diag_local(const sem_mesh *m, double h1, double h2, double *dL, cudaStream_t st);

// dinv: the Jacobi inverse of (h1, h2) for the solve's mask mode, computed by
// the caller and reused across solves (nullptr: computed here, each call)
int sem_pcg_solve_ex(const sem_mesh *m, double h1, double h2, const double *b_g, double *x_g,
                     const sem_solver_opts *opts, void *workspace, sem_solve_stats *stats, void *stream,
                     int check_every, const double *dinv = nullptr);

int sem_jacobi_inv_mode(const sem_mesh *m, double h1, double h2, int use_mask, double *dinv_g, cudaStream_t st);

// grid helpers
static inline unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 32) {
  int64_t b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}
