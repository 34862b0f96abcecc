/*
 * sem.h -- C ABI of the GB300 spectral-element hot path.
 *
 * The paper (Sec. 2.2, "NekRS") discretises each scalar field on N_e
 * hexahedral elements of order p = N with a tensor-product nodal basis on
 * Gauss-Lobatto-Legendre (GLL) points; operators are applied matrix-free as
 * dense (N+1)x(N+1) tensor contractions, carried to deformed elements by the
 * chain rule, and the stiffest substep -- the pressure Poisson solve -- is a
 * preconditioned Krylov solve. This library implements that path on one GPU:
 * mesh and GLL set-up, the local operator Ax, direct-stiffness summation
 * (gather-scatter, Q Q^T), the Jacobi preconditioner and the preconditioned
 * conjugate-gradient (PCG) solve.
 *
 * Conventions shared by every entry point
 *  - All functions return an int status: SEM_OK (0) or a negative SEM_ERR_*.
 *    sem_last_error() returns a description of the last failure on the
 *    calling thread. No C++ exception crosses this boundary.
 *  - "device" pointers are CUDA device (or managed) memory owned by the
 *    caller; "host" pointers are ordinary host memory owned by the caller.
 *    The library owns only what a handle owns (a mesh's geometry and maps)
 *    and frees it in the matching destroy call.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream. Work is enqueued on it; functions that report results
 *    to the host (sem_pcg_solve statistics, set-up) synchronise it.
 *  - Layouts. An E-vector holds one value per local node, element-major:
 *    index l = e (N+1)^3 + i + (N+1) j + (N+1)^2 k for node (i,j,k) of element
 *    e, elements numbered e = ex + nelx (ey + nely ez). A U-vector holds one
 *    value per unique (global) node g, numbered lexicographically in the
 *    lattice indices (I,J,K) = (ex N + i, ey N + j, ez N + k):
 *    g = I + nx (J + ny K), nx = nelx N + 1 (nelx N if x is periodic, with I
 *    taken mod nelx N), likewise ny.
 *  - Floating-point values are IEEE binary64 unless stated otherwise.
 */
#ifndef SEM_H
#define SEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SEM_OK = 0,
  SEM_ERR_INVALID_ARG = -1,   /* bad pointer, size or option; nothing was done */
  SEM_ERR_CUDA = -2,          /* a CUDA runtime call failed (message has the CUDA error) */
  SEM_ERR_NOT_CONVERGED = -3, /* PCG hit maxit; x holds the last iterate */
  SEM_ERR_BREAKDOWN = -4,     /* PCG met p.Ap <= 0 or a non-finite scalar */
  SEM_ERR_TIMEOUT = -5,       /* PCG exceeded opts.timeout_s; x holds the last iterate */
  SEM_ERR_IO = -6,
  SEM_ERR_NOMEM = -7          /* device allocation failed */
};

/* Arithmetic used by the operator and solver kernels. */
enum {
  SEM_PREC_FP64 = 0, /* native binary64 FMA */
  SEM_PREC_DF64 = 1, /* binary64-accurate double-float: each value carried as an
                        unevaluated sum of two binary32 (hi + lo) and combined
                        with error-free transformations (Dekker 1971; Knuth's
                        TwoSum; Joldes, Muller & Popescu 2017). About 2^-44
                        relative accuracy per operator application, relative
                        to the largest value of each element. The operators
                        compute every element at the power-of-two scale of its
                        largest input (set from the binary64 exponent, exact),
                        so any finite binary64 input is accepted; input values
                        below 2^-126 times their element's largest count as
                        zero. The geometric factors, B and the Helmholtz
                        coefficients h1, h2 must lie within |x| in
                        [2^-80, 2^100] (binary32 exponent range). */
  SEM_PREC_FP32 = 2, /* binary32 (multigrid smoothing levels) */
  SEM_PREC_BF16 = 3  /* multigrid smoothing levels: geometric factors stored as
                        bfloat16; at N = 7 the operator runs on the bfloat16
                        tensor cores (two-part bfloat16 operands, binary32
                        accumulation), at other orders in binary32 */
};

typedef struct sem_mesh sem_mesh; /* opaque */

/* A structured box of nelx x nely x nelz hexahedra of order N (1 <= N <= 10,
 * the range of polynomial orders NekRS supports, Sec. 4.1).
 * Element interfaces are uniform along x and y; along z they are uniform when
 * z_stretch == 0, else follow the tanh map
 *   z_k = Lz/2 [1 + tanh(s (2k/nelz - 1)) / tanh(s)],  s = z_stretch,
 * (the paper's tangent-hyperbolic vertical stretching, Sec. 4.2). Every GLL
 * node is then displaced (deform_amp != 0) by
 *   d_c = deform_amp h_c sin(pi xh) sin(pi yh) sin(pi zh) cos(2 pi kappa_c.xh + phi_c),
 * xh = (x/Lx, y/Ly, z/Lz), h_c = L_c / nel_c, kappa_c = kappa[3c..3c+2].
 * dirichlet[] flags the faces x=0, x=Lx, y=0, y=Ly, z=0, z=Lz that carry
 * homogeneous Dirichlet conditions (ignored in periodic directions). */
typedef struct {
  int nelx, nely, nelz;
  int N;
  double Lx, Ly, Lz;
  int periodic[3];
  int dirichlet[6];
  double z_stretch;
  double deform_amp;
  double kappa[9];
  double phi[3];
} sem_box_desc;

/* Read-only views into a mesh. Device pointers stay valid until
 * sem_mesh_destroy. G is stored element-major and factor-major within an
 * element: factor f (0..5 = rr, rs, rt, ss, st, tt) of local node p of element
 * e is G[(6 e + f) (N+1)^3 + p]. */
typedef struct {
  int64_t E, n_local, n_unique;
  int N;
  double detJ_min;
  const double *X, *Y, *Z; /* device E-vectors: node coordinates */
  const double *G;         /* device: geometric factors (6 per local node)     */
  const double *B;         /* device E-vector: rho_i rho_j rho_k |J|            */
  const int32_t *l2g;      /* device E-vector: unique id of each local node     */
  const uint8_t *mask;     /* device U-vector: 1 free, 0 Dirichlet              */
  const double *mult;      /* device U-vector: number of local copies (Q^T 1)  */
} sem_mesh_info;

typedef struct {
  double tol;      /* stop at the first iteration k with ||r_k||_2 <= tol ||b||_2 */
  int maxit;       /* > 0 */
  int precision;   /* SEM_PREC_* */
  double timeout_s;/* <= 0: no limit */
  int mask_mode;   /* 0: solve on the free nodes of the mesh's Dirichlet mask;
                      1: no mask -- the pure-Neumann (singular) operator, for
                      the pressure Poisson problem; b must be orthogonal to the
                      constant vector and x is determined up to a constant */
  int initial_guess; /* 0: start from x = 0; 1: x on entry is the initial guess
                        (zero on Dirichlet nodes): r_0 = b - A x, the stopping
                        test stays ||r|| <= tol ||b||, and a guess that meets
                        it returns at once with 0 iterations */
} sem_solver_opts;

typedef struct {
  int iterations;       /* operator applications performed */
  double rel_residual;  /* ||r||_2 / ||b||_2 at exit (Euclidean, unique nodes) */
  double solve_ms;      /* wall time of the solve on the host clock */
  int status;           /* same as the return value */
} sem_solve_stats;

/* Last error text of the calling thread ("" if none). Never NULL. */
const char *sem_last_error(void);

/* Library version string. */
const char *sem_version(void);

/* Bound of the grid-wide waits inside cooperative kernels (the persistent
 * N = 1 coarse solve of the p-multigrid): a CTA waiting at a grid barrier
 * polls at most `polls` times (about 0.1 us each) and then sets an error
 * flag, every CTA leaves the kernel at its next barrier, and the calling
 * entry point returns SEM_ERR_CUDA ("a grid barrier wait exceeded its
 * limit") with the CUDA context intact. 0 restores the default, 2^24 polls
 * (about a second). The setting is process-wide and applies to launches
 * made after the call; *previous (if not NULL) receives the old value.
 * Failure detection (no counterpart in the paper, whose runs relied on
 * scheduler-level health checks, Sec. 5.2): a kernel never hangs on a CTA
 * that does not arrive. Always returns SEM_OK. */
int sem_set_grid_wait_limit(unsigned polls, unsigned *previous);

/* GLL nodes xi[N+1] (ascending, xi_0 = -1, xi_N = 1), weights
 * rho_i = 2 / (N (N+1) P_N(xi_i)^2) and derivative matrix D[(N+1)^2],
 * row-major, D[i (N+1) + j] = l_j'(xi_i), the (p+1)x(p+1) operator matrix of
 * Sec. 2.2. Host arrays, caller-owned. SEM_ERR_INVALID_ARG for N outside
 * [1, 10] or NULL pointers. */
int sem_gll(int N, double *xi, double *rho, double *D);

/* Build a box mesh on the current CUDA device: node coordinates, geometric
 * factors G (chain rule, Sec. 2.2), mass B, the local-to-unique map l2g
 * (lattice formula in the header comment), the Dirichlet mask, the
 * gather-scatter tables and multiplicities. All set-up runs in kernels on
 * `stream`; the call synchronises it. SEM_ERR_INVALID_ARG if a size is out of
 * range, the local node count exceeds 2^31 - 1, or det J <= 0 anywhere;
 * SEM_ERR_NOMEM if device memory runs out. On success *out owns all of it. */
int sem_mesh_create_box(const sem_box_desc *desc, void *stream, sem_mesh **out);

/* Free a mesh and everything it owns (NULL is accepted). */
int sem_mesh_destroy(sem_mesh *m);

/* Fill *info with sizes and device views (the mesh-information call of the
 * boundary; "_get" because the struct type carries the name sem_mesh_info). */
int sem_mesh_info_get(const sem_mesh *m, sem_mesh_info *info);

/* Audit the index tables on the host: l2g in range, l2gm = l2g on free
 * nodes and -1 on Dirichlet nodes, CSR offsets increasing from 0 to n_local,
 * the CSR permutation a permutation whose segments hold exactly the copies of
 * their node in ascending order, multiplicities equal to the copy counts.
 * SEM_ERR_INVALID_ARG names the first violation. Copies the tables to host
 * memory (synchronous). */
int sem_mesh_validate(const sem_mesh *m);

/* Deterministic assembly (on = 1) or atomic assembly (on = 0, the default).
 * The assembled operators (sem_ax_assembled*, the PCG and p-multigrid
 * solves) add each element's contribution to a unique node with FP64/FP32
 * atomics by default, so sums over a node's copies come in a run-dependent
 * order and results agree run to run only to rounding. In deterministic mode
 * they write element results to an E-vector (8 bytes per local node, owned
 * by the mesh) and sum each node's copies in ascending copy order: results
 * are bitwise reproducible, at the cost of that scratch and one more pass
 * over it. p-multigrid hierarchies take the setting of their fine mesh when
 * they are created. Applications of operators on one deterministic mesh
 * share the scratch and must not overlap on the GPU (one stream, or
 * serialised by the caller). Turning it off synchronises the device. */
int sem_mesh_set_deterministic(sem_mesh *m, int on);

/* Arithmetic route of the double-float operator at N = 7 (SEM_PREC_DF64):
 * on = 1 evaluates the 1-D tensor contractions of Sec. 2.2 exactly on the
 * fp16 tensor cores (operands cut into five 10-bit digits on a fixed-point
 * grid per element, digit products summed exactly in binary32 by level,
 * levels recombined to double-float), four warps per element through
 * shared memory; on = 2 does the r- and s-contractions the same way with one
 * warp per element entirely in registers (t-lines on the binary32 pipe) for
 * the Poisson operator (h1 = 1, h2 = 0, the masked map), allocating
 * lane-major copies of the geometry and map (about 50 B per local point)
 * and using on = 0 for other calls; on = 0 (the default) uses the
 * compensated double-float dot products on the binary32 pipe. All meet the
 * same binary64-level accuracy. Other orders always use the binary32 route.
 * Synchronises the device when on = 2 first builds its copies. */
int sem_mesh_set_tensor_cores(sem_mesh *m, int on);

/* Copy l2g (n_local int32) and mask (n_unique uint8) to host arrays; either
 * may be NULL. Synchronous. */
int sem_mesh_copy_maps(const sem_mesh *m, int32_t *l2g_host, uint8_t *mask_host);

/* Copy the gather-scatter tables to host arrays: offsets (n_unique + 1 int32)
 * and perm (n_local int32); local nodes of unique node g are
 * perm[offsets[g] .. offsets[g+1]-1], in ascending order. Synchronous. */
int sem_mesh_copy_gs_tables(const sem_mesh *m, int32_t *offsets_host, int32_t *perm_host);

/* Local Helmholtz operator on E-vectors (no summation, no mask):
 *   w_L = h1 * sum_ab D_a^T G_ab D_b u_L + h2 * B u_L
 * (Sec. 2.2 tensor-contraction form). u_L and w_L are device E-vectors of
 * n_local values and must not overlap. precision = SEM_PREC_*. */
int sem_ax_apply(const sem_mesh *m, double h1, double h2, const double *u_L, double *w_L,
                 int precision, void *stream);

/* In-place direct stiffness summation on a device E-vector:
 * v_L <- Q Q^T v_L, i.e. every local copy of a unique node receives the sum
 * of all its copies; with apply_mask != 0 Dirichlet nodes then become 0.
 * Deterministic: copies are summed in ascending local index. */
int sem_gs_op(const sem_mesh *m, double *v_L, int apply_mask, void *stream);

/* Q^T: v_g[g] = sum of the copies of g (device E-vector -> device U-vector). */
int sem_gather(const sem_mesh *m, const double *v_L, double *v_g, void *stream);

/* Q: v_L[l] = v_g[l2g[l]] (device U-vector -> device E-vector). */
int sem_scatter(const sem_mesh *m, const double *v_g, double *v_L, void *stream);

/* Assembled operator on U-vectors in one fused pass:
 *   w_g = M Q^T (h1 A_L + h2 B) Q M u_g,  M = Dirichlet mask,
 * gathering u through l2g and summing element contributions into w_g (the
 * order of the summation is not fixed, so results may differ between calls
 * in the last bits). u_g and w_g must not overlap. */
int sem_ax_assembled(const sem_mesh *m, double h1, double h2, const double *u_g, double *w_g,
                     int precision, void *stream);

/* Weak-form load vector b_g = M Q^T (B f_L): the mass-weighted, summed and
 * masked right-hand side of -lap u = f (or of a Helmholtz problem) for a
 * forcing f given at the local nodes (device E-vector in, U-vector out). */
int sem_weak_rhs(const sem_mesh *m, const double *f_L, double *b_g, void *stream);

/* Same as sem_ax_assembled but accumulating: w_g += M Q^T (h1 A_L + h2 B) Q M u_g
 * (w_g is not cleared first). */
int sem_ax_assembled_add(const sem_mesh *m, double h1, double h2, const double *u_g, double *w_g,
                         int precision, void *stream);

/* The assembled operator of sem_ax_assembled on vectors in HOST memory:
 * w_host = M Q^T (h1 A_L + h2 B_L) Q M u_host, with the host<->device copies
 * pipelined against the arithmetic. The elements are cut into `nchunks` slabs
 * of element layers along z (0: 8; clamped to [1, nelz]; 1 for N = 1 meshes
 * and meshes in deterministic mode); unique nodes are numbered plane by plane
 * in z, so a slab reads and writes only its own lattice planes. While the
 * caller's stream applies the operator to one slab, a copy-in stream brings
 * the planes of the next slab and a copy-out stream returns the planes of
 * finished slabs (both streams created and destroyed by the call).
 * u_dev, w_dev: caller-owned device scratch of n_unique doubles each
 * (w_dev ends holding the result too). u_host, w_host: n_unique doubles;
 * page-locked (pinned) host memory lets the copies overlap, pageable memory
 * works but serialises them. The call waits for work already queued on
 * `stream` and synchronises it before returning. */
int sem_ax_assembled_host(const sem_mesh *m, double h1, double h2, const double *u_host, double *w_host,
                          int precision, double *u_dev, double *w_dev, int nchunks, void *stream);

/* nsteps independent applications of the same assembled operator (Sec. 2.2)
 * on host vectors: w_host[k] = M Q^T (h1 A_L + h2 B_L) Q M u_host[k],
 * k = 0 .. nsteps - 1, pipelined across the applications: the copy-in of
 * application k + 1, the operator of application k (on `stream`) and the
 * copy-out of application k - 1 overlap, each copy moving a whole vector
 * (a copy-in and a copy-out stream are created and destroyed by the call).
 * u_host, w_host: arrays of nsteps pointers to n_unique doubles each (pinned
 * host memory lets the copies overlap); the w_host vectors must not overlap
 * any u_host vector still to be read. u_dev2, w_dev2: caller-owned device
 * scratch of 2 n_unique doubles each (double buffers). The call waits for
 * work already queued on `stream`, returns after the last copy-out, and
 * rejects NULL pointers, a negative count, misaligned or identical device
 * buffers, an unknown precision or a mesh on another device
 * (SEM_ERR_INVALID_ARG). nsteps = 0 does nothing. */
int sem_ax_assembled_host_batch(const sem_mesh *m, double h1, double h2, int nsteps,
                                const double *const *u_host, double *const *w_host, int precision,
                                double *u_dev2, double *w_dev2, void *stream);

/* Masked inverse of the assembled diagonal of h1 A + h2 B (the Jacobi
 * preconditioner, including the D_ii D_jj G_rs cross terms at element
 * boundaries): dinv_g[g] = mask[g] / (Q^T diag_L)[g]. Device U-vector out. */
int sem_jacobi_inv(const sem_mesh *m, double h1, double h2, double *dinv_g, void *stream);

/* Number of bytes of device workspace sem_pcg_solve needs for this mesh. */
int sem_pcg_workspace_bytes(const sem_mesh *m, size_t *bytes);

/* Jacobi-preconditioned CG for (h1 A + h2 B) x = b on the free unique nodes,
 * from x0 = 0 (or from the guess in x_g when opts.initial_guess = 1), textbook
 * Hestenes-Stiefel recurrences; stops after the first iteration k with
 * ||r_k||_2 <= tol ||b||_2 (k = 0 when a guess already meets it). b_g, x_g:
 * device U-vectors (b must vanish on Dirichlet nodes; x is 0 there on exit
 * when starting from 0; a guess keeps its Dirichlet values, which the
 * operator ignores). workspace: device
 * memory of sem_pcg_workspace_bytes() bytes, 256-byte aligned, caller-owned.
 * Returns SEM_OK, SEM_ERR_NOT_CONVERGED, SEM_ERR_BREAKDOWN or SEM_ERR_TIMEOUT
 * (stats filled in every case) or an argument/CUDA error. */
int sem_pcg_solve(const sem_mesh *m, double h1, double h2, const double *b_g, double *x_g,
                  const sem_solver_opts *opts, void *workspace, sem_solve_stats *stats,
                  void *stream);

/* ------------------------------------------------------------------------
 * p-multigrid preconditioned flexible CG. Sec. 2.2: NekRS preconditions its
 * pressure Poisson solve with p-multigrid and 4th-kind Chebyshev-accelerated
 * smoothers, running most preconditioner work in FP32. Here: levels of
 * decreasing order on the same elements (each re-discretised on its own GLL
 * points with the same box description), element-wise tensor-product
 * Lagrange prolongation P and restriction R = P^T, 4th-kind Chebyshev-Jacobi
 * smoothing (Lottes 2022 recurrence) in binary32 (geometry in binary32 or
 * bfloat16), lambda_max from power iteration on D^{-1}A started from the
 * alternating lattice vector (-1)^(I+J+K), and a binary64-accurate
 * (double-float operator) Jacobi-PCG solve on the coarsest level. The outer iteration is flexible CG (Polak-Ribiere beta)
 * with the fine operator in the precision of the solver options.
 * ------------------------------------------------------------------------ */
typedef struct sem_pmg sem_pmg; /* opaque; owns its level meshes and scratch */

typedef struct {
  int nlevels;            /* 2..4 */
  int orders[4];          /* orders[0] = the fine mesh's N, strictly decreasing, >= 1 */
  int smoother_precision; /* the mixed-precision preconditioner of Sec. 2.2:
                             SEM_PREC_FP32: binary32 vectors, geometry and arithmetic;
                             SEM_PREC_BF16: binary32 vectors, bfloat16 geometry; at
                               N = 7 the operator runs on the bfloat16 tensor cores
                               (two-part bfloat16 operands, binary32 accumulation,
                               about 2^-15 relative), at other orders in binary32;
                             SEM_PREC_DF64: every smoothing level in binary64 vectors
                               with the binary64-accurate double-float operator (the
                               same V-cycle at full precision, to measure what the
                               lower precision saves) */
  int cheb_degree;        /* Chebyshev degree (operator applications per smoothing), >= 1 */
  double lambda_safety;   /* factor on the power-iteration estimate of lambda_max (e.g. 1.1) */
  int power_its;          /* power iterations (e.g. 20) */
  double coarse_tol;      /* relative tolerance of the coarsest-level solve */
  int coarse_maxit;
  int mask_mode;          /* 0: the mesh's Dirichlet mask; 1: pure Neumann (all levels
                             unmasked, constant null space; for the pressure) */
} sem_pmg_opts;

/* Build the hierarchy for the operator h1 A + h2 B on mesh m (which must
 * outlive it). Level meshes are created with the description of m at the
 * coarser orders. Synchronises the stream. */
int sem_pmg_create(const sem_mesh *m, double h1, double h2, const sem_pmg_opts *opts, void *stream,
                   sem_pmg **out);

/* lambda_max estimate of D^{-1}A on level l (after the safety factor). */
int sem_pmg_lambda(const sem_pmg *p, int level, double *lambda);

/* One V-cycle: z_g ~ A^{-1} r_g on the fine level (device U-vectors, binary64
 * in and out; r_g should vanish on Dirichlet nodes). */
int sem_pmg_vcycle(sem_pmg *p, const double *r_g, double *z_g, void *stream);

/* Prolongation (level l+1 -> l) and restriction (l -> l+1) of binary64
 * device U-vectors, for tests of the transfer operators. */
int sem_pmg_prolong(sem_pmg *p, int level, const double *uc_g, double *uf_g, void *stream);
int sem_pmg_restrict(sem_pmg *p, int level, const double *rf_g, double *rc_g, void *stream);

/* The smoothing operator of level l (l below the coarsest), as the V-cycle
 * applies it: w_g = M Q^T (h1 A_L + h2 B_L) Q M u_g with the hierarchy's h1,
 * h2, in the level's smoother precision (binary32 vectors for FP32 and BF16:
 * u_g is converted to binary32 on the way in, w_g back to binary64; at
 * N = 7 BF16 is the bfloat16 tensor-core operator). u_g, w_g: device
 * U-vectors of level l's mesh, binary64, not overlapping. For tests of the
 * level operators. */
int sem_pmg_level_apply(sem_pmg *p, int level, const double *u_g, double *w_g, void *stream);

/* Flexible CG preconditioned by one V-cycle per iteration, from x0 = 0 or, with
 * opts.initial_guess = 1, from the guess in x_g (r_0 = M b - A x_g); stops after
 * the first iteration with ||r||_2 <= tol ||b||_2 (opts.mask_mode must equal the
 * hierarchy's mask_mode; for mask_mode 1, b must be orthogonal to constants;
 * opts.precision selects the fine operator: SEM_PREC_FP64 or SEM_PREC_DF64). */
int sem_pmg_pcg_solve(sem_pmg *p, const double *b_g, double *x_g, const sem_solver_opts *opts,
                      sem_solve_stats *stats, void *stream);

int sem_pmg_destroy(sem_pmg *p);

/* ------------------------------------------------------------------------
 * Rayleigh-Benard convection time step (Boussinesq equations, Sec. 4.1,
 * Eqs. (1)-(3); periodic x, y and isothermal no-slip plates, Sec. 4.4).
 * The paper names no splitting scheme; the step is the BDF2/EXT2 high-order
 * splitting in weak form:
 *   explicit (t^n, GLL collocation): N_T = -u.grad T, N_u = -(u.grad)u + T z,
 *     wall term W = nu sum_walls (phi n . curl curl u), EXT X* = a1 X^n + a2 X^{n-1};
 *   T:  (b0/dt B + kappa A) T^{n+1} = Q^T B[(b1 T^n + b2 T^{n-1})/dt + N_T*],
 *       T = 1 - z/Lz on the plates (lifting), kappa = 1/sqrt(Ra Pr);
 *   p:  A p = Q^T[(grad phi, f*)] - W*, f* = (b1 u^n + b2 u^{n-1})/dt + N_u*,
 *       pure Neumann, right-hand side and p with zero mean;
 *   u:  (b0/dt B + nu A) u^{n+1} = M Q^T[B (f* - grad p)], u = 0 on the plates,
 *       nu = sqrt(Pr/Ra).
 * The first step uses history levels equal to the initial state. Explicit
 * terms are binary64 kernels; the five solves are sem_pcg_solve, from x0 = 0
 * or (extrapolate = 1, every step after the first) from 2 x^n - x^{n-1}
 * (extrapolate = 2: temperature and velocity from 3 x^n - 3 x^{n-1} + x^{n-2}
 * from the third step on).
 * ------------------------------------------------------------------------ */
typedef struct sem_rbc sem_rbc; /* opaque; owns its fields and scratch */

typedef struct {
  double Ra, Pr, dt;
  double tol;     /* relative residual of every solve */
  int maxit;      /* per solve */
  int precision;  /* SEM_PREC_FP64 or SEM_PREC_DF64: the operator inside the solves and the
                     explicit terms (gradients, weak divergence, H Tb; double-float for DF64) */
  int pressure_pmg; /* 1: pressure by the p-multigrid flexible CG (pure Neumann
                       hierarchy N -> N/2 -> ... -> 1, binary32 smoothing), the
                       paper's choice of preconditioner; 0: Jacobi-PCG */
  int extrapolate;  /* 1: every step after the first starts its solves from the
                       extrapolation 2 x^n - x^{n-1} of the two previous
                       solutions (T - Tb, p, u, v, w); the stopping test is
                       unchanged. The paper does not describe initial guesses;
                       this is the scheme's own second-order extrapolation.
                       2: the same, except that from the third step on the
                       temperature and velocity solves start from the
                       third-order extrapolation 3 x^n - 3 x^{n-1} + x^{n-2}
                       (the state then holds u^{n-2} and T^{n-2} too, in its
                       snapshots as well); the pressure keeps 2 p^n - p^{n-1}.
                       0: every solve starts from 0. Other values are rejected
                       with SEM_ERR_INVALID_ARG. */
} sem_rbc_params;

typedef struct {
  int step;                  /* steps completed */
  int iters_T, iters_p, iters_u[3];
  double step_ms;            /* host wall time of the step */
  int status;                /* SEM_OK or SEM_ERR_NOT_CONVERGED (a solve hit maxit) */
  double ms_explicit, ms_T, ms_p, ms_u; /* host wall time of the phases: explicit terms and
                                           wall term, temperature, pressure, velocity */
} sem_step_stats;

typedef struct {
  double *u, *v, *w, *T, *p; /* device U-vectors of the current state (owned by the handle) */
  int64_t n_unique;
  int step;
  double *u_prev, *v_prev, *w_prev; /* the velocity one step earlier (zero before the first step) */
} sem_rbc_view;

/* Create the state on mesh m (which must outlive it): u = 0, T = 1 - z/Lz
 * plus T_pert_g (device U-vector, added on the free nodes; NULL for none),
 * p = 0. The mesh must have Dirichlet plates at z = 0 and z = Lz and be
 * periodic (or walled on both sides) in x and y. Synchronises the stream. */
int sem_rbc_create(const sem_mesh *m, const sem_rbc_params *prm, const double *T_pert_g, void *stream,
                   sem_rbc **out);

/* Advance one BDF2/EXT2 step; fills *st. Returns SEM_OK, SEM_ERR_NOT_CONVERGED
 * (the step completed but a solve hit maxit) or an error. */
int sem_bdf_ext_step(sem_rbc *s, sem_step_stats *st, void *stream);

/* Device views of the current fields (valid until the next step or destroy). */
int sem_rbc_fields(const sem_rbc *s, sem_rbc_view *view);

int sem_rbc_destroy(sem_rbc *s);

/* State snapshots for checkpoint/restart. The state after a step is u, v, w,
 * their previous level, T, T^{n-1}, p, the previous wall term, p^{n-1}, with
 * extrapolate = 2 also u, v, w and T two steps earlier (U-vectors),
 * the previous advection terms of T, u, v, w (E-vectors) and the step
 * counter; every other array is rebuilt each step. Restoring a snapshot and
 * stepping again reproduces the original run bit for bit when the mesh is in
 * deterministic mode (sem_mesh_set_deterministic), otherwise to rounding.
 * sem_rbc_state_bytes: size of a snapshot: a header of eight int64 (step,
 * n_unique, n_local, E, N, format version 2, the bits of dt, 1 when the
 * levels two steps earlier are held else 0) then the arrays.
 * sem_rbc_save_state / sem_rbc_load_state: copy to / from a caller-owned
 * device buffer of that size; both synchronise the stream. Loading a
 * snapshot whose header differs in anything but the step (another mesh, dt
 * or format) returns SEM_ERR_INVALID_ARG. */
int sem_rbc_state_bytes(const sem_rbc *s, size_t *bytes);
int sem_rbc_save_state(const sem_rbc *s, void *dev_buf, void *stream);
int sem_rbc_load_state(sem_rbc *s, const void *dev_buf, void *stream);

/* The same snapshot in a file: the 8 bytes "SEMRBC01", the snapshot, then
 * its FNV-1a 64-bit checksum (little-endian). sem_rbc_load returns SEM_ERR_IO
 * for a missing, truncated or corrupted file or one whose header differs in
 * anything but the step, and then leaves the state unchanged. Both use the
 * default stream. */
int sem_rbc_save(const sem_rbc *s, const char *path);
int sem_rbc_load(sem_rbc *s, const char *path);

/* ------------------------------------------------------------------------
 * Temperature transport with a prescribed velocity history and its discrete
 * adjoint. The step is the temperature update of sem_bdf_ext_step (Sec. 4.1,
 * Eq. (2); BDF2/EXT2 of Sec. 2.2, BDF1/EXT1 at n = 0, lifting Tb = 1 - z/Lz)
 * with the velocity u^n given as data:
 *   T^{n+1} = Tb + H^{-1} M [Q^T B((b1 Q T^n + b2 Q T^{n-1})/dt + a1 N^n + a2 N^{n-1}) - Q^T H_L Q Tb],
 *   N^n = -(u^n . grad)(Q T^n),  H = kappa A + (b0/dt) B.
 * With u frozen, T^K is affine in T^0, and the transposed step gives the
 * exact gradient of a linear functional of T^K. The paper has no adjoint;
 * these calls add differentiation of its temperature step.
 * U-vectors: n_unique doubles; E-vectors: n_local doubles; all device
 * arrays, caller-owned. Every call synchronises the stream.
 * ------------------------------------------------------------------------ */
typedef struct sem_tadv sem_tadv; /* opaque; owns its scratch */

typedef struct {
  double kappa;  /* diffusivity (1/sqrt(Ra Pr) for the Boussinesq scaling) */
  double dt;
  double tol;    /* relative residual of each Helmholtz solve */
  int maxit;
  int precision; /* SEM_PREC_FP64 or SEM_PREC_DF64: the operator in the solves, the forward
                    step's gradient and H Tb (as in sem_bdf_ext_step of the same precision) */
} sem_tadv_params;

/* The mesh must have Dirichlet plates at z = 0 and z = Lz. */
int sem_tadv_create(const sem_mesh *m, const sem_tadv_params *prm, void *stream, sem_tadv **out);
int sem_tadv_destroy(sem_tadv *t);

/* A_b (the quadrature of 1 over the bottom plate) and the lifting Tb
 * (device U-vector owned by the handle). Either output may be NULL. */
int sem_tadv_info(const sem_tadv *t, double *area, const double **Tb);

/* Forward step n >= 0. u[3]: host array of three device U-vectors (u^n).
 * Tn: T^n; Tnm1, NTnm1: T^{n-1} (U) and N^{n-1} (E), ignored at n = 0.
 * Writes Tnp1 (U) and NTn = N^n (E); *iters (may be NULL) gets the PCG
 * iterations. Tnp1 must not alias an input. Returns SEM_OK,
 * SEM_ERR_NOT_CONVERGED (the step completed with maxit iterations) or an
 * error. */
int sem_tadv_step(sem_tadv *t, int n, const double *const u[3], const double *Tn, const double *Tnm1,
                  const double *NTnm1, double *Tnp1, double *NTn, int *iters, void *stream);

/* Reverse of step n: with psi = H^{-1} M g_np1 and phi = B Q psi,
 *   g_n   += Q^T [(b1/dt) phi + a1 L_n^T phi],
 *   g_nm1 += Q^T [(b2/dt) phi + a2 L_{n-1}^T phi]     (n > 0 only),
 * L_n = -(u^n . grad), so g_n is dJ/dT^n for J linear in T^K once every
 * later step has been reversed. u_n: velocity u^n; u_nm1: u^{n-1} (NULL at
 * n = 0). At n = 0 the Dirichlet entries of g_n are set to zero: g_0 is then
 * the gradient with respect to the free values of T^0. Returns like
 * sem_tadv_step. */
int sem_tadv_adjoint_step(sem_tadv *t, int n, const double *const u_n[3], const double *const u_nm1[3],
                          const double *g_np1, double *g_n, double *g_nm1, int *iters, void *stream);

/* Bottom-plate Nusselt number of the U-vector T (a host double):
 *   Nu_b = -(1/A_b) sum over the bottom-face nodes of rho_i rho_j |x_r x x_s| dT/dz,
 * dT/dz from the element-local derivatives; 1 for T = 1 - z/Lz. */
int sem_tadv_nusselt(sem_tadv *t, const double *T, double *nu, void *stream);

/* c = scale * dNu_b/dT (U-vector; Nu_b is linear in T, so Nu_b(T) = c.T at
 * scale 1). */
int sem_tadv_nusselt_grad(sem_tadv *t, double scale, double *c, void *stream);

/* ------------------------------------------------------------------------
 * In-situ slice rendering (the paper's in-situ scenes, Sec. 5.3 and the
 * figures of Sec. 4.5: temperature slices through the plate boundary layers
 * and vertical slices with iso-levels, rendered from GPU-resident data; here
 * as CUDA kernels into a caller-owned device image, no graphics API).
 * ------------------------------------------------------------------------ */
typedef struct {
  int axis;          /* plane normal: 0 (x = coord), 1 (y = coord), 2 (z = coord) */
  double coord;      /* 0 <= coord <= L[axis], in the undeformed box (on a deformed mesh the
                        plane of the reference lattice) */
  int width, height; /* pixels along the two other axes in increasing order
                        (axis 0: y, z; 1: x, z; 2: x, y); 1 .. 32768 each */
  double vmin, vmax; /* colour-map range, vmax > vmin */
  int n_iso;         /* 0 .. 8 contour levels */
  double iso[8];
} sem_slice_desc;

/* Render the unique-node field u_g (device, n_unique doubles) on the slice.
 * Pixel (px, py) is centred at ((px + 1/2) L_first / width, (py + 1/2)
 * L_second / height); row 0 is the low end; both outputs are row-major
 * [py][px], caller-owned device memory: values (width * height binary32, the
 * SEM polynomial of the element containing the pixel centre: normal-direction
 * sum in binary64, in-plane sum in binary32) and rgba (width * height * 4
 * bytes: piecewise-linear cool-warm colour map of (v - vmin) / (vmax - vmin)
 * clamped to [0, 1], blue (59, 76, 192) - grey (221, 221, 221) - red
 * (180, 4, 38), each channel rounded half up; NaN magenta; black where the
 * sign of v - level changes towards the right or upper neighbour). Allocates
 * a small table per call; synchronises the stream. */
int sem_render_slice(const sem_mesh *m, const double *u_g, const sem_slice_desc *desc, float *values,
                     uint8_t *rgba, void *stream);

/* The overview scene: iso-surfaces of a field in perspective, the box walls
 * behind them. The field (u_g, device, n_unique doubles) is resampled at the
 * cell centres of a grid[0] x grid[1] x grid[2] grid of the undeformed box
 * (each value the SEM polynomial there, binary32) into `volume` (caller-owned
 * device, [grid[2]][grid[1]][grid[0]] floats). Pinhole camera: f = target -
 * eye, r = f x up, u = r x f (normalised); pixel (px, py) looks along f +
 * s_x r + s_y u, s_x = (2 (px + 1/2)/width - 1) tan(fov/2) width/height,
 * s_y = (2 (py + 1/2)/height - 1) tan(fov/2) (row 0 at the bottom). Each ray
 * enters the box at t0 and leaves at t1 and is sampled every h = min(L_d /
 * grid[d]) from t0 with trilinear interpolation of the grid; the first sample
 * interval where v - level changes sign for some level is the hit, at the
 * linearly interpolated t. depth (width * height floats) = t, or -1 without
 * a hit; rgba = the colour map of sem_render_slice at the level times
 * 1 - (t - t_near)/(2 (t_far - t_near)) clamped to [1/2, 1] (nearest and
 * farthest box corner), rays through the box without a hit the colour map of
 * their last sample times 0.35, rays missing the box white. Allocates a small
 * table per call; synchronises the stream. */
typedef struct {
  double eye[3], target[3], up[3];
  double fov_deg;    /* vertical field of view, (0, 179) degrees */
  int width, height; /* 1 .. 16384 */
  int grid[3];       /* resampling grid, 1 .. 2048 per axis */
  double vmin, vmax; /* colour-map range, vmax > vmin */
  int n_iso;         /* 1 .. 4 levels */
  double iso[4];
} sem_scene_desc;

int sem_render_scene(const sem_mesh *m, const double *u_g, const sem_scene_desc *desc, float *volume,
                     float *depth, uint8_t *rgba, void *stream);

/* Write a host RGBA image (row 0 = low end) as a binary PPM (RGB, top row =
 * high end). SEM_ERR_IO if the file cannot be written. */
int sem_write_ppm(const char *path, const uint8_t *rgba_host, int width, int height);

/* ------------------------------------------------------------------------
 * Multi-rank partition (host only). Sec. 2.2: one rank per GPU; shared
 * surface values are summed across ranks. Rank r of P owns the element
 * planes ez in [r nelz/P, (r+1) nelz/P), i.e. elements [e_begin, e_end) in
 * the element numbering of this header. Direct stiffness summation then is a
 * rank-local Q Q^T plus a sum, over the ranks sharing it, of the partial sums
 * at each interface node (a unique node that another rank also holds).
 * ------------------------------------------------------------------------ */
/* Element range of a rank and the number of its interface nodes.
 * SEM_ERR_INVALID_ARG unless 1 <= nranks <= nelz and 0 <= rank < nranks. */
int sem_partition_info(const sem_box_desc *desc, int nranks, int rank, int64_t *e_begin, int64_t *e_end,
                       int64_t *n_interface);

/* The rank's interface nodes (unique ids, ascending) into gids[n_interface]
 * and, if nshare is not NULL, the number of ranks holding each. */
int sem_partition_interface(const sem_box_desc *desc, int nranks, int rank, int64_t *gids, int32_t *nshare);

/* The rank's exchange partners, for summing interface partial sums pairwise
 * instead of over all ranks: the other ranks q that share interface nodes
 * with it, ascending, into peers[i] = q and counts[i] = the number of nodes
 * shared with q (both arrays hold at least nranks - 1 entries, or are NULL
 * to count only), and their number into *npeers. Every node of an element-
 * slab partition is held by at most two ranks, so a node's full sum is the
 * rank's own partial sum plus the one partner's. Same argument checks as
 * sem_partition_info; NULL npeers is SEM_ERR_INVALID_ARG. */
int sem_partition_peers(const sem_box_desc *desc, int nranks, int rank, int32_t *peers, int64_t *counts,
                        int32_t *npeers);

/* The unique ids (ascending) that rank shares with peer, into
 * gids[counts[i]] from sem_partition_peers. Both ranks of a pair get the same
 * list in the same order, so their buffers of partial sums line up with no
 * exchange of indices. A peer that shares nothing writes nothing.
 * SEM_ERR_INVALID_ARG if peer is out of range or equals rank, or gids is NULL. */
int sem_partition_peer_nodes(const sem_box_desc *desc, int nranks, int rank, int peer, int64_t *gids);

/* The rank's surface elements, for overlapping the exchange with interior
 * work (Sec. 2.2: update the elements on the subdomain surface, start the
 * exchange of their shared values, update the interior elements, then finish
 * the sums with what arrived). Writes the ids (ascending) of the elements
 * that touch an interface node into elems (if not NULL; at most
 * 2 nelx nely entries) and their number into *n_surface. Every
 * contribution to an interface node comes from these elements, so the
 * interface partial sums are complete after the surface pass. Same argument
 * checks as sem_partition_info; NULL n_surface is SEM_ERR_INVALID_ARG. */
int sem_partition_surface(const sem_box_desc *desc, int nranks, int rank, int64_t *elems, int64_t *n_surface);

/* ------------------------------------------------------------------------
 * One rank's share of the element-slab partition on its GPU (Sec. 2.2: one
 * MPI rank per GPU; the gather-scatter sums shared surface values across
 * ranks, and the exchange is overlapped with the work on interior elements:
 * surface elements first, start the exchange, interior elements, finish).
 *
 * The rank holds a slab mesh: its element planes of the box, in the box's
 * element order, with the slab's own unique numbering (lattice planes
 * p0 N .. p1 N of the box, numbered like a box of that height: no periodic
 * wrap in z; the Dirichlet faces of the box where the slab reaches them).
 * Its vectors are U-vectors of that slab mesh. The communication between
 * ranks is the caller's, through two callbacks, so any transport (MPI,
 * NCCL host staging, gloo, a test harness) can carry it; the library never
 * blocks on another rank inside a kernel.
 * ------------------------------------------------------------------------ */
typedef struct sem_part sem_part; /* opaque; owns its slab mesh, lists and buffers */

/* Exchange: buf (host memory) holds this rank's partial sums at its
 * interface nodes, n of them, in the order of sem_partition_interface
 * (ascending unique id of the box). On return buf must hold, for each node,
 * the sum of the partial sums of every rank that holds it (the same value
 * on every rank). Return 0 on success; anything else ends the calling entry
 * point with SEM_ERR_IO. Called from the calling host thread only. */
typedef int (*sem_exchange_fn)(double *buf, int64_t n, void *user);

/* All-reduce: replace vals[0..n-1] by their sums over all ranks (same
 * order of summation on every rank, so that every rank takes the same
 * decisions). Return 0 on success, else the entry point returns SEM_ERR_IO. */
typedef int (*sem_allreduce_fn)(double *vals, int n, void *user);

typedef struct {
  const sem_mesh *mesh;   /* the slab mesh (owned by the partition; usable with the
                             operator, gather-scatter and solver entry points) */
  int64_t e_begin, e_end; /* the slab's elements in the box's numbering */
  int64_t n_surface;      /* elements touching an interface node */
  int64_t n_interior;     /* the other elements of the slab */
  int64_t n_interface;    /* interface nodes (exchanged values per application) */
  int64_t n_unique;       /* unique nodes of the slab mesh (the length of its vectors) */
} sem_part_info_t;

/* Build rank `rank` of `nranks` (the plan of sem_partition_info): its slab
 * mesh, surface and interior element lists, interface node list, inner-
 * product weights (1 / number of ranks holding the node) and buffers (pinned
 * host staging for the exchange, a second stream for the interior
 * elements). Same argument checks as sem_partition_info. Synchronises. */
int sem_part_create(const sem_box_desc *desc, int nranks, int rank, void *stream, sem_part **out);
int sem_part_destroy(sem_part *p);
int sem_part_info(const sem_part *p, sem_part_info_t *info);

/* The box's unique id of every unique node of the slab mesh, into
 * gids_host[n_unique] (host). */
int sem_part_global_ids(const sem_part *p, int64_t *gids_host);

/* The assembled operator over a list of elements only:
 * w_g += M Q_e^T (h1 A_e + h2 B_e) Q_e M u_g summed over e in elems
 * (device int32[n_elems], element ids of mesh m), atomic assembly. The
 * building block of the overlapped schedule; u_g, w_g are U-vectors of m.
 * SEM_ERR_INVALID_ARG for a bad list length or precision. */
int sem_ax_assembled_elems(const sem_mesh *m, double h1, double h2, const double *u_g, double *w_g,
                           const int32_t *elems, int64_t n_elems, int precision, void *stream);

/* w = M Q^T (h1 A + h2 B) Q M u on the rank's nodes, with complete sums at
 * the interface: surface elements on `stream`, their interface values
 * staged to the host and passed to ex(...) while the interior elements run
 * on the partition's second stream, the returned sums written back, the
 * streams joined. u, w: U-vectors of the slab mesh (device). The call
 * returns once the exchange is done; the rest is queued on `stream`. */
int sem_part_ax(sem_part *p, double h1, double h2, const double *u, double *w, int precision,
                sem_exchange_fn ex, void *user, void *stream);

/* Jacobi-PCG over the partition: the same iteration as sem_pcg_solve (x0 =
 * 0, stop at the first ||r|| <= tol ||b||), each operator application
 * sem_part_ax, the Jacobi diagonal summed over the ranks like the operator,
 * inner products over the rank's nodes with shared nodes weighted by one
 * over the number of ranks holding them, summed by ar(...). b, x: U-vectors
 * of the slab mesh; b must be zero on Dirichlet nodes and agree across ranks
 * on shared nodes. opts.mask_mode must be 0. Every rank returns the same
 * iteration count and status. Returns like sem_pcg_solve, or SEM_ERR_IO
 * when a callback fails. */
int sem_part_pcg_solve(sem_part *p, double h1, double h2, const double *b, double *x, const sem_solver_opts *opts,
                       sem_solve_stats *stats, sem_exchange_fn ex, sem_allreduce_fn ar, void *user, void *stream);

/* Jacobi-PCG like sem_pcg_solve, for callers that cannot allocate device
 * memory themselves -- for example a host program or plug-in whose device
 * memory is owned entirely by another framework's allocator, or a loop that
 * must not allocate once it is running. This entry point has no counterpart
 * in the paper; it exists only for such callers.
 *
 * It allocates nothing: its workspace is a fixed 64 MiB array in the
 * library's own device memory (sem_pcg_noalloc_capacity() bytes), which every
 * GPU that loads the library holds until the process exits. That bounds the
 * mesh to about 2.1 million unique nodes (4 vectors of n_unique doubles plus
 * a few kilobytes of partial sums); a larger mesh is rejected with
 * SEM_ERR_INVALID_ARG and a message giving both sizes. The caller still owns
 * b_g and x_g, as for sem_pcg_solve, and the mesh must belong to the current
 * device.
 *
 * The first call on each device looks up the array's device address (once,
 * with that device current, and again after a device reset gives the device
 * a new context); make that first call before any CUDA stream capture. All calls share the one array and every call re-initialises what
 * it reads, so results do not depend on earlier calls; but calls whose work
 * overlaps on the GPU (different streams, or different host threads on one
 * device) race on the array and must be serialised by the caller.
 * Returns the same codes as sem_pcg_solve. */
int sem_pcg_solve_noalloc(const sem_mesh *m, double h1, double h2, const double *b_g, double *x_g,
                          const sem_solver_opts *opts, sem_solve_stats *stats, void *stream);

/* Size in bytes of the fixed workspace of sem_pcg_solve_noalloc. */
size_t sem_pcg_noalloc_capacity(void);

#ifdef __cplusplus
}
#endif
#endif /* SEM_H */
