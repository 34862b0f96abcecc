"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds workload descriptions (mesh sizes, seeds) and the random
draws the workloads need. It holds none of the spectral-element arithmetic:
node coordinates, geometric factors, index maps and operators are computed
independently by each side from these parameters.

Workloads (all N = 7, i.e. 8^3 Gauss-Lobatto-Legendre points per hexahedron,
the polynomial order the paper uses for its Ra = 1e6 and Ra = 1e8 runs,
Table "Details of the simulations with Gamma = 4"):

* ``poisson_4``: unit cube of 4^3 undeformed elements, Dirichlet on all faces,
  manufactured u = sin(pi x) sin(pi y) sin(pi z), Jacobi-PCG to 1e-10.
* ``ax_gs_64``: unit cube of 64^3 elements (134,217,728 local points), every
  GLL node displaced by a smooth seeded sinusoidal deformation of amplitude
  0.1 h, input field uniform[-1, 1] per unique node.
* ``rbc_32``: 32^3 elements, tanh-stretched toward the plates (stretch 2.0),
  periodic in x and y, Ra = 1e8, Pr = 0.7.
* ``pmg_48``: the ``ax_gs_64`` construction at 48^3 elements.
* ``adjoint_16``: 16^3 elements, Ra = 1e7, Pr = 1.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Tuple

import numpy as np

DEFORM_SEED = 1      # seed of the mesh-deformation wave numbers and phases
FIELD_SEED = 0       # seed of the uniform[-1, 1] input field
RBC_PERT_SEED = 2    # seed of the temperature perturbation


@dataclasses.dataclass(frozen=True)
class BoxWorkload:
    """A structured box of hexahedral spectral elements.

    ``dirichlet`` lists the faces carrying homogeneous Dirichlet conditions as
    six flags (x=0, x=L, y=0, y=L, z=0, z=L). ``z_stretch`` = 0 means uniform
    element spacing in z; s > 0 selects the tanh interface map. ``deform_amp``
    is the sinusoidal displacement amplitude in units of the element size.
    """
    name: str
    nel: Tuple[int, int, int]
    N: int = 7
    L: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    periodic: Tuple[int, int, int] = (0, 0, 0)
    dirichlet: Tuple[int, int, int, int, int, int] = (1, 1, 1, 1, 1, 1)
    z_stretch: float = 0.0
    deform_amp: float = 0.0
    deform_seed: Optional[int] = None

    @property
    def E(self) -> int:
        return self.nel[0] * self.nel[1] * self.nel[2]

    @property
    def n_local(self) -> int:
        return self.E * (self.N + 1) ** 3

    @property
    def n_unique(self) -> int:
        n = 1
        for d in range(3):
            n *= self.nel[d] * self.N + (0 if self.periodic[d] else 1)
        return n

    @property
    def dofs(self) -> int:
        """Grid points counted as E * N^3, the convention of the paper's
        Table "Details of the simulations with Gamma = 4"."""
        return self.E * self.N ** 3

    def with_nel(self, nel, name=None) -> "BoxWorkload":
        return dataclasses.replace(self, nel=tuple(nel), name=name or self.name)


POISSON_4 = BoxWorkload("poisson_4", (4, 4, 4))
AX_GS_64 = BoxWorkload("ax_gs_64", (64, 64, 64), deform_amp=0.1, deform_seed=DEFORM_SEED)
RBC_32 = BoxWorkload("rbc_32", (32, 32, 32), periodic=(1, 1, 0),
                     dirichlet=(0, 0, 0, 0, 1, 1), z_stretch=2.0)
PMG_48 = BoxWorkload("pmg_48", (48, 48, 48), deform_amp=0.1, deform_seed=DEFORM_SEED)
ADJOINT_16 = BoxWorkload("adjoint_16", (16, 16, 16), periodic=(1, 1, 0),
                         dirichlet=(0, 0, 0, 0, 1, 1))

# the ax_gs_64 construction at 32^3 elements (16.8 M local points, geometry
# 0.8 GB > L2): the small case used for detailed kernel profiles
AX_GS_32 = AX_GS_64.with_nel((32, 32, 32), name="ax_gs_32")

WORKLOADS = {w.name: w for w in (POISSON_4, AX_GS_64, RBC_32, PMG_48, ADJOINT_16, AX_GS_32)}


def deformation_params(seed: Optional[int]):
    """Wave numbers kappa[c][d] in {1, 2} and phases phi[c] in [0, 2 pi) of the
    sinusoidal deformation, one set per coordinate c. ``None`` gives zeros."""
    if seed is None:
        return np.zeros((3, 3), dtype=np.float64), np.zeros(3, dtype=np.float64)
    rng = np.random.default_rng(seed)
    kappa = rng.integers(1, 3, size=(3, 3)).astype(np.float64)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=3)
    return kappa, phi


def unique_field(n_unique: int, seed: int = FIELD_SEED) -> np.ndarray:
    """uniform[-1, 1] FP64 value per unique node."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=n_unique)


def perturbation(n_unique: int, amp: float = 1e-3, seed: int = RBC_PERT_SEED) -> np.ndarray:
    """amp * uniform[-1, 1] per unique node (the RBC initial perturbation)."""
    rng = np.random.default_rng(seed)
    return amp * rng.uniform(-1.0, 1.0, size=n_unique)
