"""Oracle of the p-multigrid preconditioned flexible CG (TEST INFRASTRUCTURE ONLY).

Sec. 2.2: NekRS preconditions its pressure Poisson solve with p-multigrid,
using 4th-kind Chebyshev acceleration of its smoothers, and runs most of the
preconditioner in FP32 to save bandwidth. Readings (the paper gives no
algorithmic detail):

* levels: the same elements at orders N_0 > N_1 > ... (7 -> 3 -> 1), each
  level's operator re-discretised on its own GLL points with the same mesh
  mapping (coordinates evaluated at the level's nodes);
* prolongation P: element-wise tensor-product Lagrange interpolation from the
  coarse to the fine GLL points (continuity is preserved, so a fine unique
  value is any of its identical local copies); restriction R = P^T;
* smoother: Chebyshev polynomial of the 4th kind in D^{-1} A (Jacobi), degree
  k, with the recurrence of Lottes (2022), "Optimal polynomial smoothers for
  multigrid V-cycles"; lambda_max from power iteration on D^{-1} A started
  from the alternating lattice vector (-1)^(I+J+K), times a safety factor;
* coarsest level: Jacobi-PCG to a relative tolerance;
* V-cycle: pre-smooth from zero, restrict the residual, recurse, prolong and
  add, post-smooth;
* outer iteration: flexible CG (Polak-Ribiere form of beta), x0 = 0, stop
  after the first iteration with ||r|| <= tol ||b||.
Everything here is binary64.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import Mesh, apply_assembled, box_mesh, gather_sum, jacobi_inv, pcg, scatter


def lagrange_matrix(xc: np.ndarray, xf: np.ndarray) -> np.ndarray:
    """J[i, m] = l_m(xf_i): values of the Lagrange basis on the nodes xc at
    the points xf (interpolation from xc to xf)."""
    J = np.ones((len(xf), len(xc)))
    for m in range(len(xc)):
        for j in range(len(xc)):
            if j != m:
                J[:, m] *= (xf - xc[j]) / (xc[m] - xc[j])
    return J


def apply_tensor(J: np.ndarray, v: np.ndarray, E: int) -> np.ndarray:
    """Per element: (J x J x J) applied to a (nc,nc,nc) tile, local order
    i + n j + n^2 k (i fastest)."""
    nf, nc = J.shape
    t = v.reshape(E, nc, nc, nc)  # [e, k, j, i]
    t = np.einsum("ai,ekji->ekja", J, t)
    t = np.einsum("bj,ekja->ekba", J, t)
    t = np.einsum("ck,ekba->ecba", J, t)
    return t.reshape(E * nf ** 3)


@dataclass
class Level:
    m: Mesh
    dinv: np.ndarray
    lam: float
    mk: np.ndarray


class PMG:
    def __init__(self, box: dict, orders=(7, 3, 1), h1=1.0, h2=0.0, degree=2, safety=1.1, power_its=20,
                 coarse_tol=1e-10, coarse_maxit=2000):
        self.h1, self.h2, self.degree = h1, h2, degree
        self.coarse_tol, self.coarse_maxit = coarse_tol, coarse_maxit
        self.levels: List[Level] = []
        for N in orders:
            m = box_mesh(N=N, **box)
            dinv = jacobi_inv(m, h1, h2)
            mk = m.mask.astype(np.float64)
            lev = Level(m, dinv, 0.0, mk)
            lev.lam = safety * self.lambda_max(lev, power_its)
            self.levels.append(lev)
        self.J = [lagrange_matrix(self.levels[l + 1].m.xi, self.levels[l].m.xi) for l in range(len(orders) - 1)]

    def A(self, l: int, v: np.ndarray) -> np.ndarray:
        return apply_assembled(self.levels[l].m, v, self.h1, self.h2)

    def lambda_max(self, lev: Level, its: int) -> float:
        m = lev.m
        n = [m.nel[d] * m.N + (0 if m.periodic[d] else 1) for d in range(3)]
        g = np.arange(m.n_unique)
        I, Jl, K = g % n[0], (g // n[0]) % n[1], g // (n[0] * n[1])
        v = np.where((I + Jl + K) % 2 == 0, 1.0, -1.0) * lev.mk
        lam = 0.0
        for _ in range(its):
            w = lev.dinv * apply_assembled(m, v, self.h1, self.h2)
            lam = float(np.sqrt(np.dot(w, w) / np.dot(v, v)))
            v = w / np.sqrt(np.dot(w, w))
        return lam

    def prolong(self, l: int, uc: np.ndarray) -> np.ndarray:
        """coarse level l+1 -> fine level l (unique vectors)."""
        mf, mc = self.levels[l].m, self.levels[l + 1].m
        vf = apply_tensor(self.J[l], scatter(mc, uc), mf.E)
        return gather_sum(mf, vf) / mf.mult

    def restrict(self, l: int, rf: np.ndarray) -> np.ndarray:
        """fine level l -> coarse level l+1: R = P^T."""
        mf, mc = self.levels[l].m, self.levels[l + 1].m
        vf = scatter(mf, rf / mf.mult)
        return gather_sum(mc, apply_tensor(self.J[l].T, vf, mf.E))

    def smooth(self, l: int, b: np.ndarray, x: Optional[np.ndarray] = None) -> np.ndarray:
        """4th-kind Chebyshev-Jacobi, degree k (Lottes 2022)."""
        lev = self.levels[l]
        lam, k = lev.lam, self.degree
        if x is None:
            x = np.zeros_like(b)
            r = b.copy()
        else:
            x = x.copy()
            r = b - self.A(l, x)
        d = (4.0 / (3.0 * lam)) * lev.dinv * r
        for i in range(1, k + 1):
            x = x + d
            if i == k:
                break
            r = r - self.A(l, d)
            d = ((2 * i - 1) / (2 * i + 3)) * d + ((8 * i + 4) / ((2 * i + 3) * lam)) * lev.dinv * r
        return x

    def vcycle(self, b: np.ndarray, l: int = 0) -> np.ndarray:
        if l == len(self.levels) - 1:
            lev = self.levels[l]
            return pcg(lev.m, b * lev.mk, self.h1, self.h2, tol=self.coarse_tol, maxit=self.coarse_maxit).x
        x = self.smooth(l, b)
        r = b - self.A(l, x)
        xc = self.vcycle(self.restrict(l, r), l + 1)
        x = x + self.prolong(l, xc)
        return self.smooth(l, b, x)


@dataclass
class FCGResult:
    x: np.ndarray
    iterations: int
    rel_residual: float
    converged: bool
    history: list


def fcg(pm: PMG, b: np.ndarray, tol: float = 1e-8, maxit: int = 200) -> FCGResult:
    """Flexible CG with the V-cycle preconditioner on the finest level."""
    A = lambda v: pm.A(0, v)  # noqa: E731
    mk = pm.levels[0].mk
    b = np.asarray(b, dtype=np.float64) * mk
    x = np.zeros_like(b)
    r = b.copy()
    bn = float(np.linalg.norm(b))
    hist = []
    if bn == 0.0:
        return FCGResult(x, 0, 0.0, True, hist)
    z = pm.vcycle(r) * mk
    p = z.copy()
    rz = float(np.dot(r, z))
    for it in range(1, maxit + 1):
        w = A(p)
        alpha = rz / float(np.dot(p, w))
        x += alpha * p
        r -= alpha * w
        rn = float(np.linalg.norm(r))
        hist.append(rn / bn)
        if rn <= tol * bn:
            return FCGResult(x, it, rn / bn, True, hist)
        zn = pm.vcycle(r) * mk
        beta = float(np.dot(r, zn - z)) / rz
        rz = float(np.dot(r, zn))
        p = zn + beta * p
        z = zn
    return FCGResult(x, maxit, hist[-1], False, hist)
