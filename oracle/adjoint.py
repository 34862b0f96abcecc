"""Oracle of the temperature step with frozen velocity, its discrete adjoint,
and the bottom-wall Nusselt functional (TEST INFRASTRUCTURE ONLY).

Equation: the temperature equation of Sec. 4.1, Eq. (2), dT/dt + u.grad T =
kappa lap T, kappa = 1/sqrt(Ra Pr), on the Rayleigh-Benard box of Sec. 4.4
(T = 1 on z = 0, T = 0 on z = Lz), discretised exactly as in oracle.rbc
(BDF1/EXT1 first step, then BDF2/EXT2; Dirichlet lifting 1 - z/Lz).

Reading (the paper has no adjoint; the workload names the functional): the
velocity history u^0..u^{K-1} is frozen data from a forward run, so T^K is
affine in T^0 and the discrete adjoint gives the exact gradient of
  Nu_b(T) = -(1 / A_b) sum over bottom faces of rho_i rho_j |x_r x x_s| dT/dz,
A_b = the same quadrature of 1 (equals 1 for the conduction state T = 1 - z;
the volume form of Sec. 4.5 is not used). dT/dz is the element-local
derivative at the bottom-face nodes.

Forward step n (x = T^n, y = T^{n-1}, L_n = -u^n.grad, local):
  T^{n+1} = Tb + H^{-1} M [Q^T B((b1 Qx + b2 Qy)/dt + a1 L_n Qx + a2 L_{n-1} Qy) - H_L Tb]
Adjoint: with psi = H^{-1} M g^{n+1} and phi = B Q psi,
  g^n     += Q^T [(b1/dt) phi + a1 L_n^T phi],
  g^{n-1} += Q^T [(b2/dt) phi + a2 L_{n-1}^T phi],
  L^T phi = -sum_a D_a^T (sum_c dr_a/dx_c u_c phi)   (transpose of -u.grad).
"""
from __future__ import annotations

from typing import List, Optional

import numpy as np

from . import Mesh, ax_local, gather_sum, lib, pcg, scatter
from .rbc import coefficients, geometry, grad


def advect(m: Mesh, g, uL: List[np.ndarray], fL: np.ndarray) -> np.ndarray:
    """L f = -u . grad f at the local nodes."""
    gf = grad(m, g, fL)
    return -(uL[0] * gf[0] + uL[1] * gf[1] + uL[2] * gf[2])


def advect_t(m: Mesh, g, uL: List[np.ndarray], phi: np.ndarray) -> np.ndarray:
    """L^T phi = -sum_a D_a^T (sum_c dr_a/dx_c u_c phi), local."""
    v = np.stack([-sum(g.R[a, c] * uL[c] * phi for c in range(3)) for a in range(3)]).ravel()
    out = np.zeros(m.n_local)
    lib().or_ref_div_t(m.E, m.N, np.ascontiguousarray(m.D.ravel()), v, out)
    return out


def bottom_weights(m: Mesh, g) -> np.ndarray:
    """E-vector of rho_i rho_j |x_r x x_s| at the bottom-face nodes (k = 0 of
    the elements with ez = 0), zero elsewhere."""
    n = m.N + 1
    w = np.zeros(m.n_local)
    e = np.arange(m.E)
    ez = e // (m.nel[0] * m.nel[1])
    I, Jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pts = (I + n * Jj).ravel()
    wts = (m.rho[I] * m.rho[Jj]).ravel()
    for el in np.nonzero(ez == 0)[0]:
        l = el * n ** 3 + pts
        area = np.cross(g.J[:, 0, l].T, g.J[:, 1, l].T)
        w[l] = wts * np.linalg.norm(area, axis=1)
    return w


def nusselt_bottom(m: Mesh, g, T: np.ndarray) -> float:
    w = bottom_weights(m, g)
    dTdz = grad(m, g, scatter(m, T))[2]
    return float(-np.dot(w, dTdz) / w.sum())


def nusselt_bottom_grad(m: Mesh, g) -> np.ndarray:
    """c with Nu_b(T) = c . T (the functional is linear in T)."""
    w = bottom_weights(m, g)
    # Nu = -(1/A) sum_l w_l sum_a R_a2(l) (D_a Q T)_l = Q^T[-(1/A) sum_a D_a^T (R_a2 w)] . T
    v = np.stack([-(g.R[a, 2] * w) / w.sum() for a in range(3)]).ravel()
    out = np.zeros(m.n_local)
    lib().or_ref_div_t(m.E, m.N, np.ascontiguousarray(m.D.ravel()), v, out)
    return gather_sum(m, out)


class TAdv:
    """Temperature steps with a prescribed velocity history."""

    def __init__(self, m: Mesh, kappa: float, dt: float, tol: float = 1e-13, maxit: int = 5000):
        self.m, self.kappa, self.dt, self.tol, self.maxit = m, kappa, dt, tol, maxit
        self.g = geometry(m)
        Tb = np.zeros(m.n_unique)
        Tb[m.l2g] = 1.0 - m.Z / m.L[2]
        self.Tb = Tb
        self.mk = m.mask.astype(np.float64)

    def step(self, n: int, u: List[np.ndarray], Tn: np.ndarray, Tnm1: Optional[np.ndarray],
             NTnm1: Optional[np.ndarray]):
        """T^{n+1} and the local N_T^n from T^n, T^{n-1}, N_T^{n-1}."""
        m, dt = self.m, self.dt
        b0, b1, b2, a1, a2 = coefficients(n)
        uL = [scatter(m, c) for c in u]
        TL = scatter(m, Tn)
        NT = advect(m, self.g, uL, TL)
        if n == 0:
            Tnm1, NTnm1 = Tn, NT
        TpL = scatter(m, Tnm1)
        TbL = scatter(m, self.Tb)
        rhs = gather_sum(m, m.B * ((b1 * TL + b2 * TpL) / dt + a1 * NT + a2 * NTnm1))
        rhs = rhs - gather_sum(m, ax_local(m, TbL, self.kappa, b0 / dt))
        r = pcg(m, self.mk * rhs, self.kappa, b0 / dt, tol=self.tol, maxit=self.maxit)
        return self.Tb + r.x, NT

    def forward(self, T0: np.ndarray, us: List[List[np.ndarray]]) -> np.ndarray:
        Tn, Tnm1, NTnm1 = T0, None, None
        for n, u in enumerate(us):
            Tnp1, NT = self.step(n, u, Tn, Tnm1, NTnm1)
            Tnm1, Tn, NTnm1 = Tn, Tnp1, NT
        return Tn

    def adjoint(self, gK: np.ndarray, us: List[List[np.ndarray]]) -> np.ndarray:
        """dJ/dT^0 (free nodes) for J = gK . T^K."""
        m, dt = self.m, self.dt
        K = len(us)
        g = [np.zeros(m.n_unique) for _ in range(K + 1)]
        g[K] = gK.copy()
        for n in range(K - 1, -1, -1):
            b0, b1, b2, a1, a2 = coefficients(n)
            psi = pcg(m, self.mk * g[n + 1], self.kappa, b0 / dt, tol=self.tol, maxit=self.maxit).x
            phi = m.B * scatter(m, psi)
            uL = [scatter(m, c) for c in us[n]]
            g[n] += gather_sum(m, (b1 / dt) * phi + a1 * advect_t(m, self.g, uL, phi))
            if n >= 1:
                upL = [scatter(m, c) for c in us[n - 1]]
                g[n - 1] += gather_sum(m, (b2 / dt) * phi + a2 * advect_t(m, self.g, upL, phi))
        return g[0] * self.mk
