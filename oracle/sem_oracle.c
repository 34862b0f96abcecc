/*
 * Plain FP64 CPU oracle of the spectral-element hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and
 * its Python binding) may include, link or call this file. Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg use it.
 *
 * It follows the paper's description of NekRS (Sec. 2.2): N_e hexahedral
 * elements of order p = N with a tensor-product nodal basis on
 * Gauss-Lobatto-Legendre (GLL) points, operators evaluated matrix-free as
 * tensor contractions with the (N+1)x(N+1) derivative matrix, carried to
 * deformed elements by the chain rule. Everything the paper leaves to its
 * cited textbook (Deville, Fischer & Mund 2002) is the textbook definition,
 * written out loop by loop with no blocking, fusion or reordering:
 *
 *   - GLL nodes xi_i: -1, +1 and the roots of P_N'; weights
 *     rho_i = 2 / (N (N+1) P_N(xi_i)^2); derivative matrix D_ij = l_j'(xi_i).
 *   - geometry: J_ca = dx_c/dr_a by D applied to the node coordinates,
 *     G_ab = rho_i rho_j rho_k |J| sum_c (dr_a/dx_c)(dr_b/dx_c), B = rho|J|.
 *   - local operator w_L = h1 * sum_ab D_a^T G_ab D_b u_L + h2 * B u_L.
 *   - direct stiffness summation Q Q^T through the global lattice index.
 *
 * Every function here is pinned in the tests against closed forms, library
 * routines or brute force (see tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXN 16

/* P_N(x) and P_N'(x) by the three-term recurrence, long double. */
static void legendre_pd(int N, long double x, long double *P, long double *dP) {
  long double p0 = 1.0L, p1 = x, dp0 = 0.0L, dp1 = 1.0L;
  if (N == 0) { *P = 1.0L; *dP = 0.0L; return; }
  for (int k = 2; k <= N; ++k) {
    long double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    long double dp2 = dp0 + (2 * k - 1) * p1; /* P_k' = P_{k-2}' + (2k-1) P_{k-1} */
    p0 = p1; p1 = p2; dp0 = dp1; dp1 = dp2;
  }
  *P = p1; *dP = dp1;
}

/* GLL nodes, weights and derivative matrix (row-major D[i*(N+1)+j] = l_j'(xi_i)).
 * Interior nodes: Newton on P_N' from Chebyshev-Gauss-Lobatto guesses, with
 * P_N'' from Legendre's equation (1-x^2) P'' = 2x P' - N(N+1) P.
 * Returns 0, or -1 for N outside [1, MAXN-1]. */
int or_gll(int N, double *xi, double *rho, double *D) {
  if (N < 1 || N >= MAXN) return -1;
  long double x[MAXN], P[MAXN];
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i <= N; ++i) {
    long double t = -cosl(pi * i / N);
    if (i > 0 && i < N) {
      for (int it = 0; it < 100; ++it) {
        long double p, dp;
        legendre_pd(N, t, &p, &dp);
        long double ddp = (2.0L * t * dp - N * (N + 1) * p) / (1.0L - t * t);
        long double step = dp / ddp;
        t -= step;
        if (fabsl(step) < 1e-19L) break;
      }
    }
    x[i] = t;
  }
  x[0] = -1.0L; x[N] = 1.0L;
  /* enforce the exact symmetry xi_{N-i} = -xi_i */
  for (int i = 0; i <= N / 2; ++i) { long double a = 0.5L * (x[N - i] - x[i]); x[i] = -a; x[N - i] = a; }
  if (N % 2 == 0) x[N / 2] = 0.0L;
  for (int i = 0; i <= N; ++i) {
    long double dp;
    legendre_pd(N, x[i], &P[i], &dp);
    xi[i] = (double)x[i];
    rho[i] = (double)(2.0L / (N * (N + 1) * P[i] * P[i]));
  }
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N; ++j) {
      long double d;
      if (i != j) d = P[i] / (P[j] * (x[i] - x[j]));
      else if (i == 0) d = -(long double)N * (N + 1) / 4.0L;
      else if (i == N) d = (long double)N * (N + 1) / 4.0L;
      else d = 0.0L;
      D[i * (N + 1) + j] = (double)d;
    }
  return 0;
}

/* Local node (e; i,j,k) of a box of nelx*nely*nelz elements, e = ex + nelx(ey + nely ez),
 * local index l = e n^3 + i + n j + n^2 k (n = N+1), has lattice indices
 * (I,J,K) = (ex N + i, ey N + j, ez N + k). Its unique id is
 * g = I + nx (J + ny K) with nx = nelx N + 1 (nelx N and I mod nelx N when
 * the direction is periodic). */
void or_lattice_l2g(int nelx, int nely, int nelz, int N, const int *periodic, int64_t *l2g) {
  const int n = N + 1;
  const int64_t nx = (int64_t)nelx * N + (periodic[0] ? 0 : 1);
  const int64_t ny = (int64_t)nely * N + (periodic[1] ? 0 : 1);
  for (int ez = 0; ez < nelz; ++ez)
    for (int ey = 0; ey < nely; ++ey)
      for (int ex = 0; ex < nelx; ++ex) {
        int64_t e = ex + (int64_t)nelx * (ey + (int64_t)nely * ez);
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              int64_t I = (int64_t)ex * N + i, J = (int64_t)ey * N + j, K = (int64_t)ez * N + k;
              if (periodic[0]) I %= (int64_t)nelx * N;
              if (periodic[1]) J %= (int64_t)nely * N;
              if (periodic[2]) K %= (int64_t)nelz * N;
              l2g[e * n * n * n + i + n * j + n * n * k] = I + nx * (J + ny * K);
            }
      }
}

/* Dirichlet mask per unique node: 0 on a flagged face, 1 elsewhere.
 * faces = {x=0, x=L, y=0, y=L, z=0, z=L}; ignored in periodic directions. */
void or_lattice_mask(int nelx, int nely, int nelz, int N, const int *periodic, const int *faces,
                     uint8_t *mask) {
  int64_t nd[3] = {(int64_t)nelx * N + (periodic[0] ? 0 : 1), (int64_t)nely * N + (periodic[1] ? 0 : 1),
                   (int64_t)nelz * N + (periodic[2] ? 0 : 1)};
  for (int64_t K = 0; K < nd[2]; ++K)
    for (int64_t J = 0; J < nd[1]; ++J)
      for (int64_t I = 0; I < nd[0]; ++I) {
        int64_t idx[3] = {I, J, K};
        int m = 1;
        for (int d = 0; d < 3; ++d) {
          if (periodic[d]) continue;
          if (faces[2 * d] && idx[d] == 0) m = 0;
          if (faces[2 * d + 1] && idx[d] == nd[d] - 1) m = 0;
        }
        mask[I + nd[0] * (J + nd[1] * K)] = (uint8_t)m;
      }
}

/* Element interface coordinates along one direction: uniform, or the tanh
 * map z_k = L/2 [1 + tanh(s(2k/n - 1)) / tanh(s)] when s > 0. */
static double interface_coord(int k, int nel, double L, double s) {
  if (s > 0.0) return 0.5 * L * (1.0 + tanh(s * (2.0 * k / nel - 1.0)) / tanh(s));
  return L * (double)k / (double)nel;
}

/* GLL node coordinates of a box mesh, E-vector order. The reference
 * coordinate xi maps linearly into each element,
 * x = x_e (1 - xi)/2 + x_{e+1} (1 + xi)/2, then every node is displaced by
 *   d_c = amp h_c sin(pi xh) sin(pi yh) sin(pi zh) cos(2 pi kappa_c . xh + phi_c),
 * xh = x / L (normalised position), h_c = L_c / nel_c. */
static void box_coords_element(int nelx, int nely, int nelz, int N, const double *L, double z_stretch, double amp,
                               const double *kappa, const double *phi, const double *xi, int64_t e, double *X,
                               double *Y, double *Z) {
  const int n = N + 1;
  const int nel[3] = {nelx, nely, nelz};
  const double pi = 3.14159265358979323846;
  int eidx[3] = {(int)(e % nelx), (int)((e / nelx) % nely), (int)(e / ((int64_t)nelx * nely))};
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        int node[3] = {i, j, k};
        double x[3];
        for (int d = 0; d < 3; ++d) {
          double s = (d == 2) ? z_stretch : 0.0;
          double a = interface_coord(eidx[d], nel[d], L[d], s);
          double b = interface_coord(eidx[d] + 1, nel[d], L[d], s);
          double t = xi[node[d]];
          x[d] = a * (0.5 * (1.0 - t)) + b * (0.5 * (1.0 + t));
        }
        double xo[3] = {x[0], x[1], x[2]};
        if (amp != 0.0) {
          double xh[3] = {x[0] / L[0], x[1] / L[1], x[2] / L[2]};
          double bump = sin(pi * xh[0]) * sin(pi * xh[1]) * sin(pi * xh[2]);
          for (int c = 0; c < 3; ++c) {
            double arg = 2.0 * pi * (kappa[3 * c] * xh[0] + kappa[3 * c + 1] * xh[1] + kappa[3 * c + 2] * xh[2]) + phi[c];
            xo[c] = x[c] + amp * (L[c] / nel[c]) * bump * cos(arg);
          }
        }
        int p = i + n * j + n * n * k;
        X[p] = xo[0]; Y[p] = xo[1]; Z[p] = xo[2];
      }
}

/* GLL node coordinates of a box mesh, E-vector order. The reference
 * coordinate xi maps linearly into each element,
 * x = x_e (1 - xi)/2 + x_{e+1} (1 + xi)/2, then every node is displaced by
 *   d_c = amp h_c sin(pi xh) sin(pi yh) sin(pi zh) cos(2 pi kappa_c . xh + phi_c),
 * xh = x / L (normalised position), h_c = L_c / nel_c. */
void or_box_coords(int nelx, int nely, int nelz, int N, const double *L, double z_stretch, double amp,
                   const double *kappa, const double *phi, const double *xi, double *X, double *Y,
                   double *Z) {
  const int64_t n3 = (int64_t)(N + 1) * (N + 1) * (N + 1);
  const int64_t E = (int64_t)nelx * nely * nelz;
  for (int64_t e = 0; e < E; ++e)
    box_coords_element(nelx, nely, nelz, N, L, z_stretch, amp, kappa, phi, xi, e, X + e * n3, Y + e * n3, Z + e * n3);
}

/* The same coordinates for a list of elements only (ne elements, output
 * packed element after element), for spot checks of very large meshes. */
void or_box_coords_subset(int nelx, int nely, int nelz, int N, const double *L, double z_stretch, double amp,
                          const double *kappa, const double *phi, const double *xi, const int64_t *elems,
                          int64_t ne, double *X, double *Y, double *Z) {
  const int64_t n3 = (int64_t)(N + 1) * (N + 1) * (N + 1);
  for (int64_t t = 0; t < ne; ++t)
    box_coords_element(nelx, nely, nelz, N, L, z_stretch, amp, kappa, phi, xi, elems[t], X + t * n3, Y + t * n3,
                       Z + t * n3);
}

/* Geometric factors. G is stored factor-major: G[a*nL + l], a = 0..5 for
 * (rr, rs, rt, ss, st, tt); B[l] = rho_i rho_j rho_k |J|. Returns the minimum
 * of det J over all nodes (the caller rejects meshes with det J <= 0). */
double or_geom(int64_t E, int N, const double *D, const double *rho, const double *X, const double *Y,
               const double *Z, double *G, double *B) {
  const int n = N + 1;
  const int64_t nL = E * n * n * n;
  const double *xc[3] = {X, Y, Z};
  double detmin = INFINITY;
  for (int64_t e = 0; e < E; ++e)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int64_t base = e * n * n * n;
          double J[3][3]; /* J[c][a] = dx_c / dr_a */
          for (int c = 0; c < 3; ++c) {
            double dr = 0, ds = 0, dt = 0;
            for (int m = 0; m < n; ++m) {
              dr += D[i * n + m] * xc[c][base + m + n * j + n * n * k];
              ds += D[j * n + m] * xc[c][base + i + n * m + n * n * k];
              dt += D[k * n + m] * xc[c][base + i + n * j + n * n * m];
            }
            J[c][0] = dr; J[c][1] = ds; J[c][2] = dt;
          }
          double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
                     - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
                     + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
          if (det < detmin) detmin = det;
          /* inverse: R[a][c] = dr_a / dx_c = cofactor(J)[c][a] / det */
          double R[3][3];
          R[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
          R[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
          R[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
          R[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
          R[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
          R[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
          R[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
          R[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
          R[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
          double w = rho[i] * rho[j] * rho[k] * det;
          int64_t l = base + i + n * j + n * n * k;
          const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
          for (int f = 0; f < 6; ++f) {
            double s = 0;
            for (int c = 0; c < 3; ++c) s += R[pa[f]][c] * R[pb[f]][c];
            G[f * nL + l] = w * s;
          }
          B[l] = w;
        }
  return detmin;
}

/* Local (unassembled) Helmholtz operator w_L = h1 A_L u_L + h2 B u_L with
 * A_L = [D_r^T D_s^T D_t^T] G [D_r; D_s; D_t], element by element.
 * G may be NULL only when h1 == 0; B may be NULL only when h2 == 0. */
void or_ax_local(int64_t E, int N, const double *D, const double *G, const double *B, double h1,
                 double h2, const double *u, double *w) {
  const int n = N + 1, n3 = n * n * n;
  const int64_t nL = E * n3;
#pragma omp parallel
  {
    double ur[MAXN * MAXN * MAXN], us[MAXN * MAXN * MAXN], ut[MAXN * MAXN * MAXN];
#pragma omp for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
      const double *ue = u + e * n3;
      double *we = w + e * n3;
      int64_t base = e * n3;
      /* gradient in reference coordinates */
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            double a = 0, b = 0, c = 0;
            for (int m = 0; m < n; ++m) {
              a += D[i * n + m] * ue[m + n * j + n * n * k];
              b += D[j * n + m] * ue[i + n * m + n * n * k];
              c += D[k * n + m] * ue[i + n * j + n * n * m];
            }
            ur[i + n * j + n * n * k] = a;
            us[i + n * j + n * n * k] = b;
            ut[i + n * j + n * n * k] = c;
          }
      /* multiply by the symmetric metric G */
      if (h1 != 0.0) {
        for (int p = 0; p < n3; ++p) {
          int64_t l = base + p;
          double g00 = G[0 * nL + l], g01 = G[1 * nL + l], g02 = G[2 * nL + l];
          double g11 = G[3 * nL + l], g12 = G[4 * nL + l], g22 = G[5 * nL + l];
          double a = ur[p], b = us[p], c = ut[p];
          ur[p] = g00 * a + g01 * b + g02 * c;
          us[p] = g01 * a + g11 * b + g12 * c;
          ut[p] = g02 * a + g12 * b + g22 * c;
        }
      }
      /* transposed derivative, then the mass term */
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            double s = 0;
            if (h1 != 0.0)
              for (int m = 0; m < n; ++m) {
                s += D[m * n + i] * ur[m + n * j + n * n * k];
                s += D[m * n + j] * us[i + n * m + n * n * k];
                s += D[m * n + k] * ut[i + n * j + n * n * m];
              }
            int p = i + n * j + n * n * k;
            double v = h1 * s;
            if (h2 != 0.0) v += h2 * B[base + p] * ue[p];
            we[p] = v;
          }
    }
  }
}

/* Diagonal of the local operator h1 A_L + h2 B, element by element, from its
 * definition: diag_p = sum_ab sum_q D_a[q,p] G_ab[q] D_b[q,p]. The r-r term
 * runs over the line through p; the cross terms meet only at q = p. */
void or_diag_local(int64_t E, int N, const double *D, const double *G, const double *B, double h1,
                   double h2, double *d) {
  const int n = N + 1, n3 = n * n * n;
  const int64_t nL = E * n3;
  for (int64_t e = 0; e < E; ++e)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int64_t base = e * n3;
          int64_t l = base + i + n * j + n * n * k;
          double s = 0;
          for (int m = 0; m < n; ++m) {
            s += D[m * n + i] * D[m * n + i] * G[0 * nL + base + m + n * j + n * n * k];
            s += D[m * n + j] * D[m * n + j] * G[3 * nL + base + i + n * m + n * n * k];
            s += D[m * n + k] * D[m * n + k] * G[5 * nL + base + i + n * j + n * n * m];
          }
          s += 2.0 * D[i * n + i] * D[j * n + j] * G[1 * nL + l];
          s += 2.0 * D[i * n + i] * D[k * n + k] * G[2 * nL + l];
          s += 2.0 * D[j * n + j] * D[k * n + k] * G[4 * nL + l];
          d[l] = h1 * s + (h2 != 0.0 ? h2 * B[l] : 0.0);
        }
}

/* Q^T: vg[g] = sum over local copies l with l2g[l] = g of vL[l]. */
void or_gather_sum(int64_t nL, const int64_t *l2g, const double *vL, int64_t nU, double *vg) {
  memset(vg, 0, sizeof(double) * (size_t)nU);
  for (int64_t l = 0; l < nL; ++l) vg[l2g[l]] += vL[l];
}

/* Q: vL[l] = vg[l2g[l]]. */
void or_scatter(int64_t nL, const int64_t *l2g, const double *vg, double *vL) {
  for (int64_t l = 0; l < nL; ++l) vL[l] = vg[l2g[l]];
}

#ifdef _OPENMP
#include <omp.h>
int or_num_threads(void) { return omp_get_max_threads(); }
#else
int or_num_threads(void) { return 1; }
#endif

/* Jacobian of the isoparametric map at every node: J[(3c + a) nL + l] =
 * dx_c/dr_a (D applied to the node coordinates, as in or_geom). */
void or_jacobian(int64_t E, int N, const double *D, const double *X, const double *Y, const double *Z,
                 double *J) {
  const int n = N + 1;
  const int64_t nL = E * n * n * n;
  const double *xc[3] = {X, Y, Z};
  for (int64_t e = 0; e < E; ++e)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int64_t base = e * n * n * n, l = base + i + n * j + n * n * k;
          for (int c = 0; c < 3; ++c) {
            double dr = 0, ds = 0, dt = 0;
            for (int m = 0; m < n; ++m) {
              dr += D[i * n + m] * xc[c][base + m + n * j + n * n * k];
              ds += D[j * n + m] * xc[c][base + i + n * m + n * n * k];
              dt += D[k * n + m] * xc[c][base + i + n * j + n * n * m];
            }
            J[(3 * c + 0) * nL + l] = dr;
            J[(3 * c + 1) * nL + l] = ds;
            J[(3 * c + 2) * nL + l] = dt;
          }
        }
}

/* Reference-space derivatives of an E-vector: d[a nL + l] = (D_a f)_l,
 * a = r, s, t. */
void or_ref_grad(int64_t E, int N, const double *D, const double *f, double *d) {
  const int n = N + 1;
  const int64_t nL = E * n * n * n;
  for (int64_t e = 0; e < E; ++e)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int64_t base = e * n * n * n, l = base + i + n * j + n * n * k;
          double dr = 0, ds = 0, dt = 0;
          for (int m = 0; m < n; ++m) {
            dr += D[i * n + m] * f[base + m + n * j + n * n * k];
            ds += D[j * n + m] * f[base + i + n * m + n * n * k];
            dt += D[k * n + m] * f[base + i + n * j + n * n * m];
          }
          d[0 * nL + l] = dr;
          d[1 * nL + l] = ds;
          d[2 * nL + l] = dt;
        }
}

/* Transposed reference derivatives: out_l = sum_a (D_a^T v_a)_l for three
 * E-vectors v_r, v_s, v_t stored as v[a nL + l]. */
void or_ref_div_t(int64_t E, int N, const double *D, const double *v, double *out) {
  const int n = N + 1;
  const int64_t nL = E * n * n * n;
  for (int64_t e = 0; e < E; ++e)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int64_t base = e * n * n * n, l = base + i + n * j + n * n * k;
          double s = 0;
          for (int m = 0; m < n; ++m) {
            s += D[m * n + i] * v[0 * nL + base + m + n * j + n * n * k];
            s += D[m * n + j] * v[1 * nL + base + i + n * m + n * n * k];
            s += D[m * n + k] * v[2 * nL + base + i + n * j + n * n * m];
          }
          out[l] = s;
        }
}
