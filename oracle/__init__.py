"""Plain FP64 CPU oracle of the spectral-element hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users. The product package never
imports it, and it never imports the product package.

The numerics live in ``sem_oracle.c`` (plain loops, FP64); this module wraps
them with ctypes and adds the assembled (unique-node) operator and the
textbook preconditioned conjugate-gradient solve. Passages followed:

* Sec. 2.2 (NekRS): N_e hexahedra of order p, GLL nodal basis, matrix-free
  tensor contractions with (p+1)x(p+1) matrices, chain rule for deformed
  elements; the pressure Poisson solve is the stiffest substep and is
  preconditioned.
* Sec. 4.1, Eqs. (1)-(3): Boussinesq equations (used by the time step).
* Sec. 4.4: periodic x, y; isothermal no-slip plates; T = 1 - z initial state.

Readings where the paper is silent (Jacobi diagonal, residual norm, mesh
deformation, tanh map) are stated at each function.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sem_oracle.c")
_LIB = os.path.join(_HERE, "libsemoracle.so")

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile sem_oracle.c into libsemoracle.so (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.or_gll.argtypes = [ctypes.c_int, _dp, _dp, _dp]
        L.or_gll.restype = ctypes.c_int
        L.or_lattice_l2g.argtypes = [ctypes.c_int] * 4 + [_ip, _i64p]
        L.or_lattice_l2g.restype = None
        L.or_lattice_mask.argtypes = [ctypes.c_int] * 4 + [_ip, _ip, _u8p]
        L.or_lattice_mask.restype = None
        L.or_box_coords.argtypes = [ctypes.c_int] * 4 + [_dp, ctypes.c_double, ctypes.c_double,
                                                         _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_box_coords.restype = None
        L.or_box_coords_subset.argtypes = [ctypes.c_int] * 4 + [_dp, ctypes.c_double, ctypes.c_double,
                                                                _dp, _dp, _dp, _i64p, ctypes.c_int64, _dp, _dp, _dp]
        L.or_box_coords_subset.restype = None
        L.or_geom.argtypes = [ctypes.c_int64, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_geom.restype = ctypes.c_double
        L.or_ax_local.argtypes = [ctypes.c_int64, ctypes.c_int, _dp, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.or_ax_local.restype = None
        L.or_diag_local.argtypes = [ctypes.c_int64, ctypes.c_int, _dp, _dp, _dp, ctypes.c_double,
                                    ctypes.c_double, _dp]
        L.or_diag_local.restype = None
        L.or_gather_sum.argtypes = [ctypes.c_int64, _i64p, _dp, ctypes.c_int64, _dp]
        L.or_gather_sum.restype = None
        L.or_scatter.argtypes = [ctypes.c_int64, _i64p, _dp, _dp]
        L.or_scatter.restype = None
        L.or_jacobian.argtypes = [ctypes.c_int64, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
        L.or_jacobian.restype = None
        L.or_ref_grad.argtypes = [ctypes.c_int64, ctypes.c_int, _dp, _dp, _dp]
        L.or_ref_grad.restype = None
        L.or_ref_div_t.argtypes = [ctypes.c_int64, ctypes.c_int, _dp, _dp, _dp]
        L.or_ref_div_t.restype = None
        L.or_num_threads.argtypes = []
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().or_num_threads())


# --------------------------------------------------------------------------
# GLL basis (Sec. 2.2: nodal GLL basis, (p+1)x(p+1) operator matrices)
# --------------------------------------------------------------------------
def gll(N: int):
    """GLL nodes xi[N+1], weights rho[N+1], derivative matrix D[N+1, N+1]
    with D[i, j] = l_j'(xi_i)."""
    xi = np.zeros(N + 1)
    rho = np.zeros(N + 1)
    D = np.zeros((N + 1) * (N + 1))
    if lib().or_gll(N, xi, rho, D) != 0:
        raise ValueError(f"unsupported order N={N}")
    return xi, rho, D.reshape(N + 1, N + 1)


# --------------------------------------------------------------------------
# Box mesh (Sec. 4.4 box; tanh stretching of Sec. 4.2)
# --------------------------------------------------------------------------
@dataclass
class Mesh:
    nel: tuple
    N: int
    periodic: tuple
    dirichlet: tuple
    xi: np.ndarray
    rho: np.ndarray
    D: np.ndarray
    X: np.ndarray
    Y: np.ndarray
    Z: np.ndarray
    G: Optional[np.ndarray]
    B: Optional[np.ndarray]
    l2g: np.ndarray
    mask: np.ndarray       # per unique node, 1 = free, 0 = Dirichlet
    n_unique: int
    detJ_min: float
    L: tuple = (1.0, 1.0, 1.0)
    z_stretch: float = 0.0
    _mult: Optional[np.ndarray] = field(default=None, repr=False)

    @property
    def E(self) -> int:
        return self.nel[0] * self.nel[1] * self.nel[2]

    @property
    def n_local(self) -> int:
        return self.E * (self.N + 1) ** 3

    @property
    def mult(self) -> np.ndarray:
        """Multiplicity of each unique node: Q^T 1."""
        if self._mult is None:
            self._mult = gather_sum(self, np.ones(self.n_local))
        return self._mult


def box_mesh(nel, N=7, L=(1.0, 1.0, 1.0), periodic=(0, 0, 0), dirichlet=(1, 1, 1, 1, 1, 1),
             z_stretch=0.0, deform_amp=0.0, kappa=None, phi=None, geometry=True, coords=None) -> Mesh:
    """Build the oracle's view of a box mesh.

    Reading of the deformation (the workload names only "smooth seeded
    sinusoidal deformation of amplitude 0.1 h"): every GLL node is displaced
    by amp*h_c*sin(pi x)sin(pi y)sin(pi z)*cos(2 pi kappa_c.x + phi_c) in
    normalised coordinates; it vanishes on the boundary of the box.
    ``coords`` = (X, Y, Z) overrides the generated coordinates (tests use it
    for analytic mappings)."""
    nel = tuple(int(v) for v in nel)
    xi, rho, D = gll(N)
    E = nel[0] * nel[1] * nel[2]
    nL = E * (N + 1) ** 3
    per = np.array(periodic, dtype=np.int32)
    if coords is None:
        X, Y, Z = np.zeros(nL), np.zeros(nL), np.zeros(nL)
        kap = np.zeros(9) if kappa is None else np.ascontiguousarray(np.asarray(kappa, dtype=np.float64).ravel())
        ph = np.zeros(3) if phi is None else np.ascontiguousarray(np.asarray(phi, dtype=np.float64))
        lib().or_box_coords(nel[0], nel[1], nel[2], N, np.asarray(L, dtype=np.float64), float(z_stretch),
                            float(deform_amp), kap, ph, xi, X, Y, Z)
    else:
        X, Y, Z = (np.ascontiguousarray(c, dtype=np.float64) for c in coords)
    l2g = np.zeros(nL, dtype=np.int64)
    lib().or_lattice_l2g(nel[0], nel[1], nel[2], N, per, l2g)
    nd = [nel[d] * N + (0 if periodic[d] else 1) for d in range(3)]
    nU = nd[0] * nd[1] * nd[2]
    mask = np.zeros(nU, dtype=np.uint8)
    lib().or_lattice_mask(nel[0], nel[1], nel[2], N, per, np.asarray(dirichlet, dtype=np.int32), mask)
    G = B = None
    detmin = float("nan")
    if geometry:
        G = np.zeros(6 * nL)
        B = np.zeros(nL)
        detmin = lib().or_geom(E, N, np.ascontiguousarray(D.ravel()), rho, X, Y, Z, G, B)
        if not detmin > 0.0:
            raise ValueError(f"mesh has a non-positive Jacobian (min det J = {detmin})")
        G = G.reshape(6, nL)
    return Mesh(nel, N, tuple(periodic), tuple(dirichlet), xi, rho, D, X, Y, Z, G, B, l2g, mask, nU,
                detmin, tuple(L), float(z_stretch))


def element_subset(w, elems):
    """Coordinates, geometric factors and mass of selected elements of a
    workload's mesh (element-local quantities only), for spot checks of meshes
    too large to build whole: returns (X, Y, Z, G[6, ne*n3], B, D) packed in
    the order of ``elems``."""
    from workloads import deformation_params
    kappa, phi = deformation_params(w.deform_seed)
    xi, rho, D = gll(w.N)
    elems = np.ascontiguousarray(elems, dtype=np.int64)
    n3 = (w.N + 1) ** 3
    nL = len(elems) * n3
    X, Y, Z = np.zeros(nL), np.zeros(nL), np.zeros(nL)
    lib().or_box_coords_subset(w.nel[0], w.nel[1], w.nel[2], w.N, np.asarray(w.L, dtype=np.float64),
                               float(w.z_stretch), float(w.deform_amp), np.ascontiguousarray(kappa.ravel()),
                               np.ascontiguousarray(phi), xi, elems, len(elems), X, Y, Z)
    G = np.zeros(6 * nL)
    B = np.zeros(nL)
    lib().or_geom(len(elems), w.N, np.ascontiguousarray(D.ravel()), rho, X, Y, Z, G, B)
    return X, Y, Z, G.reshape(6, nL), B, D


def ax_local_raw(N, D, G, B, u, h1=1.0, h2=0.0):
    """Local operator on packed element data (G shaped [6, nL])."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.zeros_like(u)
    n3 = (N + 1) ** 3
    Gc = np.ascontiguousarray(G.ravel())
    Bc = np.ascontiguousarray(B)
    lib().or_ax_local(len(u) // n3, N, np.ascontiguousarray(D.ravel()), Gc.ctypes.data if h1 != 0.0 else None,
                      Bc.ctypes.data if h2 != 0.0 else None, float(h1), float(h2), u, w)
    return w


def mesh_from_workload(w, geometry=True) -> Mesh:
    """Mesh of a ``workloads.BoxWorkload``."""
    from workloads import deformation_params
    kappa, phi = deformation_params(w.deform_seed)
    return box_mesh(w.nel, w.N, w.L, w.periodic, w.dirichlet, w.z_stretch, w.deform_amp, kappa, phi,
                    geometry=geometry)


# --------------------------------------------------------------------------
# Operators
# --------------------------------------------------------------------------
def ax_local(m: Mesh, u: np.ndarray, h1: float = 1.0, h2: float = 0.0) -> np.ndarray:
    """w_L = h1 A_L u_L + h2 B u_L (local, unassembled; Sec. 2.2 tensor form)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.zeros_like(u)
    Gp = m.G.ctypes.data if (h1 != 0.0) else None
    Bp = m.B.ctypes.data if (h2 != 0.0) else None
    lib().or_ax_local(m.E, m.N, np.ascontiguousarray(m.D.ravel()), Gp, Bp, float(h1), float(h2), u, w)
    return w


def gather_sum(m: Mesh, vL: np.ndarray) -> np.ndarray:
    """Q^T v: sum of the local copies of each unique node."""
    vg = np.zeros(m.n_unique)
    lib().or_gather_sum(m.n_local, m.l2g, np.ascontiguousarray(vL, dtype=np.float64), m.n_unique, vg)
    return vg


def scatter(m: Mesh, vg: np.ndarray) -> np.ndarray:
    """Q v: copy each unique value to its local copies."""
    vL = np.zeros(m.n_local)
    lib().or_scatter(m.n_local, m.l2g, np.ascontiguousarray(vg, dtype=np.float64), vL)
    return vL


def qqt(m: Mesh, vL: np.ndarray, apply_mask: bool = False) -> np.ndarray:
    """Direct stiffness summation Q Q^T v_L (then the Dirichlet mask)."""
    vg = gather_sum(m, vL)
    if apply_mask:
        vg = vg * m.mask
    return scatter(m, vg)


def apply_assembled(m: Mesh, ug: np.ndarray, h1: float = 1.0, h2: float = 0.0) -> np.ndarray:
    """A_g u_g = M Q^T (h1 A_L + h2 B) Q M u_g with M the Dirichlet mask."""
    mk = m.mask.astype(np.float64)
    return mk * gather_sum(m, ax_local(m, scatter(m, mk * ug), h1, h2))


def diag_assembled(m: Mesh, h1: float = 1.0, h2: float = 0.0) -> np.ndarray:
    """Assembled diagonal Q^T diag(h1 A_L + h2 B) (no mask).

    Reading: the Jacobi preconditioner uses the exact assembled diagonal,
    including the G_rs D_ii D_jj cross terms at element faces."""
    d = np.zeros(m.n_local)
    Bp = m.B if m.B is not None else np.zeros(m.n_local)
    lib().or_diag_local(m.E, m.N, np.ascontiguousarray(m.D.ravel()), np.ascontiguousarray(m.G.ravel()),
                        Bp, float(h1), float(h2), d)
    return gather_sum(m, d)


def jacobi_inv(m: Mesh, h1: float = 1.0, h2: float = 0.0) -> np.ndarray:
    """Masked inverse of the assembled diagonal."""
    d = diag_assembled(m, h1, h2)
    out = np.zeros_like(d)
    free = m.mask != 0
    out[free] = 1.0 / d[free]
    return out


# --------------------------------------------------------------------------
# Manufactured Poisson problem on the unit cube (workload poisson_4)
# --------------------------------------------------------------------------
def manufactured_u(m: Mesh) -> np.ndarray:
    """u = sin(pi x) sin(pi y) sin(pi z) at the local nodes."""
    return np.sin(np.pi * m.X) * np.sin(np.pi * m.Y) * np.sin(np.pi * m.Z)


def poisson_rhs(m: Mesh) -> np.ndarray:
    """b = M Q^T (B f) with f = -lap u = 3 pi^2 u (weak form of -lap u = f)."""
    f = 3.0 * np.pi ** 2 * manufactured_u(m)
    return m.mask * gather_sum(m, m.B * f)


@dataclass
class SolveResult:
    x: np.ndarray
    iterations: int
    rel_residual: float
    converged: bool
    history: list


def pcg(m: Mesh, b: np.ndarray, h1: float = 1.0, h2: float = 0.0, tol: float = 1e-10,
        maxit: int = 1000, precond: str = "jacobi", apply=None, x0: np.ndarray = None) -> SolveResult:
    """Textbook preconditioned conjugate gradients (Hestenes-Stiefel) on the
    unique-node vectors, from x0 (zero when not given): r_0 = b - A x0.

    Reading of the stopping rule (the paper gives none): stop after the first
    iteration k with ||r_k||_2 <= tol ||b||_2, Euclidean norms over the unique
    nodes (||b||, not ||r_0||, so that an initial guess does not change what
    is solved); the iteration count is the number of operator applications."""
    A = apply or (lambda v: apply_assembled(m, v, h1, h2))
    if precond == "jacobi":
        dinv = jacobi_inv(m, h1, h2)
    elif precond == "none":
        dinv = m.mask.astype(np.float64)
    else:
        raise ValueError(precond)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    bn = float(np.sqrt(np.dot(b, b)))
    hist = []
    if bn == 0.0:
        return SolveResult(x, 0, 0.0, True, hist)
    if x0 is not None:
        x = np.array(x0, dtype=np.float64)
        r = b - A(x)
        rn0 = float(np.sqrt(np.dot(r, r)))
        if rn0 <= tol * bn:  # the guess already meets the tolerance
            return SolveResult(x, 0, rn0 / bn, True, hist)
    z = dinv * r
    p = z.copy()
    rho = float(np.dot(r, z))
    for it in range(1, maxit + 1):
        w = A(p)
        pw = float(np.dot(p, w))
        alpha = rho / pw
        x += alpha * p
        r -= alpha * w
        rn = float(np.sqrt(np.dot(r, r)))
        hist.append(rn / bn)
        if rn <= tol * bn:
            return SolveResult(x, it, rn / bn, True, hist)
        z = dinv * r
        rho1 = float(np.dot(r, z))
        beta = rho1 / rho
        rho = rho1
        p = z + beta * p
    return SolveResult(x, maxit, hist[-1], False, hist)
