"""Oracle of the BDF2/EXT2 Rayleigh-Benard time step (TEST INFRASTRUCTURE ONLY).

Equations: the non-dimensional Boussinesq system of Sec. 4.1, Eqs. (1)-(3):
    du/dt + u.grad u = -grad p + T z + sqrt(Pr/Ra) lap u,
    dT/dt + u.grad T = 1/sqrt(Ra Pr) lap T,        div u = 0,
on a box periodic in x and y with isothermal no-slip plates (Sec. 4.4):
u = 0 and T = 1 at z = 0, T = 0 at z = Lz, initial state u = 0, T = 1 - z
(Sec. 4.4) plus a seeded perturbation.

The paper gives no time-splitting scheme (it names NekRS and its pressure
Poisson solve, Sec. 2.2). Reading: the high-order splitting of the
spectral-element textbook the paper cites, in weak form, step n -> n+1:

  1. explicit terms at t^n, collocated at the GLL nodes (no dealiasing):
     N_T = -u.grad T, N_u = -(u.grad)u + T z, and the wall term
     W = nu * sum over wall faces of the surface quadrature of phi n.(curl curl u)
     (element-local derivatives); EXT2: X* = 2 X^n - X^{n-1}.
  2. temperature: (b0/dt B + kappa A) T^{n+1} = Q^T B [(2 T^n - T^{n-1}/2)/dt + N_T*]
     with the Dirichlet lifting T = (1 - z/Lz) + theta, theta = 0 on the plates.
  3. pressure: A p = Q^T [sum_a D_a^T (B sum_c (dr_a/dx_c) f*_c)] - W*,
     f* = (2 u^n - u^{n-1}/2)/dt + N_u*, no Dirichlet nodes, right-hand side
     and solution with their mean removed (the constant null space).
  4. velocity: (b0/dt B + nu A) u_c^{n+1} = M Q^T [B f*_c - B dp/dx_c], u = 0 on
     the plates.
  BDF2 (b0, b1, b2) = (3/2, 2, -1/2) on (x^{n+1}, x^n, x^{n-1}); EXT2 (2, -1);
  the first step is BDF1/EXT1 ((1, 1, 0), (1, 0)): starting BDF2 with history
  levels equal to the initial state would shift the solution by dt/3 in time
  and make the scheme first order (pinned by the temporal-order test).
All solves are the oracle's Jacobi-PCG to a caller-given tolerance.
Parity of this scheme is pinned by exact properties (conduction fixed point,
zero explicit terms at rest) and otherwise only by this oracle's own scheme.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import Mesh, ax_local, gather_sum, lib, pcg, scatter

B0, B1, B2 = 1.5, 2.0, -0.5
A1, A2 = 2.0, -1.0
FIRST = (1.0, 1.0, 0.0, 1.0, 0.0)  # BDF1/EXT1 for the first step


def coefficients(step: int):
    """(b0, b1, b2, a1, a2) of the step that starts from level `step`."""
    return FIRST if step == 0 else (B0, B1, B2, A1, A2)


@dataclass
class Geometry:
    J: np.ndarray  # [c, a, l] = dx_c / dr_a
    R: np.ndarray  # [a, c, l] = dr_a / dx_c


def geometry(m: Mesh) -> Geometry:
    nL = m.n_local
    J = np.zeros(9 * nL)
    lib().or_jacobian(m.E, m.N, np.ascontiguousarray(m.D.ravel()), m.X, m.Y, m.Z, J)
    J = J.reshape(3, 3, nL)
    R = np.linalg.inv(J.transpose(2, 0, 1)).transpose(1, 2, 0)  # inv(J)[a][c]
    return Geometry(J, np.ascontiguousarray(R))


def ref_grad(m: Mesh, f: np.ndarray) -> np.ndarray:
    d = np.zeros(3 * m.n_local)
    lib().or_ref_grad(m.E, m.N, np.ascontiguousarray(m.D.ravel()), np.ascontiguousarray(f), d)
    return d.reshape(3, m.n_local)


def grad(m: Mesh, g: Geometry, f: np.ndarray) -> np.ndarray:
    """Physical gradient at the local nodes: df/dx_c = sum_a dr_a/dx_c D_a f."""
    d = ref_grad(m, f)
    return np.stack([sum(g.R[a, c] * d[a] for a in range(3)) for c in range(3)])


def weak_div(m: Mesh, g: Geometry, f: List[np.ndarray]) -> np.ndarray:
    """sum_a D_a^T (B sum_c dr_a/dx_c f_c), local (before Q^T): (grad phi, f)."""
    v = np.stack([m.B * sum(g.R[a, c] * f[c] for c in range(3)) for a in range(3)]).ravel()
    out = np.zeros(m.n_local)
    lib().or_ref_div_t(m.E, m.N, np.ascontiguousarray(m.D.ravel()), v, out)
    return out


def curl(m: Mesh, g: Geometry, u: List[np.ndarray]) -> List[np.ndarray]:
    gu = [grad(m, g, c) for c in u]  # gu[i][j] = du_i/dx_j
    return [gu[2][1] - gu[1][2], gu[0][2] - gu[2][0], gu[1][0] - gu[0][1]]


def wall_faces(m: Mesh):
    """(direction, side) of every non-periodic face carrying the velocity
    Dirichlet condition."""
    out = []
    for d in range(3):
        if m.periodic[d]:
            continue
        for side in (0, 1):
            if m.dirichlet[2 * d + side]:
                out.append((d, side))
    return out


def wall_term(m: Mesh, g: Geometry, u: List[np.ndarray], nu: float) -> np.ndarray:
    """W = nu sum over wall faces of rho rho (+-x_a x x_b) . curl(curl u),
    gathered to unique nodes (unnormalised outward area vector)."""
    n = m.N + 1
    w = curl(m, g, curl(m, g, u))
    contrib = np.zeros(m.n_local)
    nel = m.nel
    e = np.arange(m.E)
    eidx = [e % nel[0], (e // nel[0]) % nel[1], e // (nel[0] * nel[1])]
    rho = m.rho
    idx = np.arange(n)
    for d, side in wall_faces(m):
        elems = np.nonzero(eidx[d] == (0 if side == 0 else nel[d] - 1))[0]
        a, b = [(1, 2), (2, 0), (0, 1)][d]  # tangential directions, x_a x x_b along +r_d
        I, Jj, K = np.meshgrid(idx, idx, idx, indexing="ij")
        loc = [I, Jj, K]
        sel = loc[d] == (0 if side == 0 else n - 1)
        pts = (I + n * Jj + n * n * K)[sel]
        wts = (rho[loc[a]] * rho[loc[b]])[sel]
        sign = -1.0 if side == 0 else 1.0
        for el in elems:
            l = el * n ** 3 + pts
            xa = g.J[:, a, l]
            xb = g.J[:, b, l]
            area = np.cross(xa.T, xb.T).T  # (3, npts)
            contrib[l] += nu * sign * wts * sum(area[c] * w[c][l] for c in range(3))
    return gather_sum(m, contrib)


def _pcg_helm(m: Mesh, b, h1, h2, tol, maxit, x0=None):
    return pcg(m, b, h1, h2, tol=tol, maxit=maxit, x0=x0)


def _pcg_neumann(m: Mesh, b, tol, maxit, x0=None):
    """Jacobi-PCG on the unmasked Poisson operator (constant null space)."""
    free = Mesh(m.nel, m.N, m.periodic, m.dirichlet, m.xi, m.rho, m.D, m.X, m.Y, m.Z, m.G, m.B, m.l2g,
                np.ones(m.n_unique, dtype=np.uint8), m.n_unique, m.detJ_min, m.L)

    def apply(v):
        return gather_sum(free, ax_local(free, scatter(free, v), 1.0, 0.0))

    return pcg(free, b, 1.0, 0.0, tol=tol, maxit=maxit, apply=apply, x0=x0)


@dataclass
class RBCState:
    u: List[np.ndarray]
    T: np.ndarray
    p: np.ndarray
    u_prev: Optional[List[np.ndarray]] = None
    T_prev: Optional[np.ndarray] = None
    NT_prev: Optional[np.ndarray] = None
    Nu_prev: Optional[List[np.ndarray]] = None
    W_prev: Optional[np.ndarray] = None
    p_prev: Optional[np.ndarray] = None
    step: int = 0
    iters: dict = field(default_factory=dict)
    u_prev2: Optional[List[np.ndarray]] = None  # two steps earlier (third-order guesses only)
    T_prev2: Optional[np.ndarray] = None


class RBC:
    """extrapolate: start the solves of every step after the first from the
    second-order extrapolation 2 x^n - x^{n-1} of the two previous solutions
    (the stopping test stays ||r|| <= tol ||b||). The paper does not describe
    its solvers' initial guesses; this is the extrapolation of the scheme's
    own order (EXT2), a simple form of starting from earlier solutions.
    extrapolate = 2: the temperature and velocity solves start from the
    third-order extrapolation 3 x^n - 3 x^{n-1} + x^{n-2} once three levels
    exist (from the third step; the second step uses 2 x^n - x^{n-1}); the
    pressure keeps the second-order guess (its history is not smooth enough
    for a higher order, measured on this oracle)."""

    def __init__(self, m: Mesh, Ra: float, Pr: float, dt: float, tol=1e-12, maxit=5000, extrapolate=False):
        self.extrapolate = extrapolate
        self.m = m
        self.geo = geometry(m)
        self.nu = np.sqrt(Pr / Ra)
        self.kappa = 1.0 / np.sqrt(Ra * Pr)
        self.dt = dt
        self.tol = tol
        self.maxit = maxit
        Lz = m.L[2]
        Tb = np.zeros(m.n_unique)
        Tb[m.l2g] = 1.0 - m.Z / Lz
        self.Tb = Tb

    def initial_state(self, pert: Optional[np.ndarray] = None) -> RBCState:
        m = self.m
        T = self.Tb.copy()
        if pert is not None:
            T = T + pert * m.mask
        z = np.zeros(m.n_unique)
        return RBCState([z.copy(), z.copy(), z.copy()], T, z.copy())

    def explicit(self, uL, TL):
        m, g = self.m, self.geo
        gT = grad(m, g, TL)
        NT = -(uL[0] * gT[0] + uL[1] * gT[1] + uL[2] * gT[2])
        Nu = []
        for c in range(3):
            gc = grad(m, g, uL[c])
            Nu.append(-(uL[0] * gc[0] + uL[1] * gc[1] + uL[2] * gc[2]))
        Nu[2] = Nu[2] + TL
        W = wall_term(m, g, uL, self.nu)
        return NT, Nu, W

    def step(self, s: RBCState) -> RBCState:
        m, g, dt = self.m, self.geo, self.dt
        uL = [scatter(m, c) for c in s.u]
        TL = scatter(m, s.T)
        NT, Nu, W = self.explicit(uL, TL)
        if s.step == 0:
            s.u_prev = [c.copy() for c in s.u]
            s.T_prev = s.T.copy()
            s.NT_prev, s.Nu_prev, s.W_prev = NT, Nu, W
        upL = [scatter(m, c) for c in s.u_prev]
        TpL = scatter(m, s.T_prev)
        b0, b1, b2, a1, a2 = coefficients(s.step)
        NTs = a1 * NT + a2 * s.NT_prev
        Nus = [a1 * Nu[c] + a2 * s.Nu_prev[c] for c in range(3)]
        Ws = a1 * W + a2 * s.W_prev
        mk = m.mask.astype(np.float64)
        # temperature with lifting
        TbL = scatter(m, self.Tb)
        rhsT = gather_sum(m, m.B * ((b1 * TL + b2 * TpL) / dt + NTs))
        rhsT = rhsT - gather_sum(m, (b0 / dt) * m.B * TbL) - self.kappa * gather_sum(m, ax_local(m, TbL, 1.0, 0.0))
        ex = bool(self.extrapolate) and s.step >= 1  # two earlier levels exist
        ex3 = self.extrapolate == 2 and s.step >= 2  # three earlier levels exist
        if ex3:
            x0 = mk * (3.0 * (s.T - self.Tb) - 3.0 * (s.T_prev - self.Tb) + (s.T_prev2 - self.Tb))
        else:
            x0 = mk * (2.0 * (s.T - self.Tb) - (s.T_prev - self.Tb)) if ex else None
        rT = _pcg_helm(m, mk * rhsT, self.kappa, b0 / dt, self.tol, self.maxit, x0=x0)
        T_new = self.Tb + rT.x
        # pressure
        fs = [(b1 * uL[c] + b2 * upL[c]) / dt + Nus[c] for c in range(3)]
        rhsp = gather_sum(m, weak_div(m, g, fs)) - Ws
        rhsp = rhsp - rhsp.mean()
        rp = _pcg_neumann(m, rhsp, self.tol, self.maxit, x0=(2.0 * s.p - s.p_prev) if ex else None)
        p = rp.x - rp.x.mean()
        # velocity
        gp = grad(m, g, scatter(m, p))
        u_new, its = [], []
        for c in range(3):
            rhs = mk * gather_sum(m, m.B * (fs[c] - gp[c]))
            if ex3:
                x0 = mk * (3.0 * s.u[c] - 3.0 * s.u_prev[c] + s.u_prev2[c])
            else:
                x0 = mk * (2.0 * s.u[c] - s.u_prev[c]) if ex else None
            r = _pcg_helm(m, rhs, self.nu, b0 / dt, self.tol, self.maxit, x0=x0)
            u_new.append(r.x)
            its.append(r.iterations)
        out = RBCState(u_new, T_new, p, [c.copy() for c in s.u], s.T.copy(), NT, Nu, W, s.p.copy(), s.step + 1,
                       {"T": rT.iterations, "p": rp.iterations, "u": its},
                       [c.copy() for c in s.u_prev], s.T_prev.copy())
        return out

    def divergence(self, s: RBCState) -> float:
        """max |div u| at the local nodes (element-local derivatives)."""
        m, g = self.m, self.geo
        uL = [scatter(m, c) for c in s.u]
        div = sum(grad(m, g, uL[c])[c] for c in range(3))
        return float(np.abs(div).max())
