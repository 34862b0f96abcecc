"""Pins of the oracle's discrete adjoint of the frozen-velocity temperature
steps and of the bottom-wall Nusselt functional (Sec. 4.1 Eq. (2); plates of
Sec. 4.4): Nu_b = 1 for conduction, linearity of the functional, the adjoint
against the dense Jacobian built column by column, and central finite
differences. CPU only."""
import numpy as np
import pytest

import oracle
from oracle import adjoint, rbc


def rbc_mesh(nel=(2, 2, 3), N=4, stretch=1.5):
    return oracle.box_mesh(nel, N, periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), z_stretch=stretch)


def velocities(m, K, amp=0.3, seed=4):
    rng = np.random.default_rng(seed)
    return [[amp * rng.standard_normal(m.n_unique) * m.mask for _ in range(3)] for _ in range(K)]


def test_nusselt_of_conduction_is_one():
    m = rbc_mesh()
    g = rbc.geometry(m)
    z = np.zeros(m.n_unique)
    z[m.l2g] = m.Z
    assert abs(adjoint.nusselt_bottom(m, g, 1.0 - z) - 1.0) < 1e-13
    # twice the gradient -> twice the flux; and the gradient vector is the functional
    assert abs(adjoint.nusselt_bottom(m, g, 2.0 * (1.0 - z)) - 2.0) < 1e-13
    c = adjoint.nusselt_bottom_grad(m, g)
    T = np.random.default_rng(1).standard_normal(m.n_unique)
    assert abs(np.dot(c, T) - adjoint.nusselt_bottom(m, g, T)) < 1e-12 * np.abs(c).sum()


def test_adjoint_equals_dense_jacobian():
    m = rbc_mesh((2, 2, 2), 3, 1.0)
    K, kappa, dt = 4, 0.05, 0.01
    ta = adjoint.TAdv(m, kappa, dt)
    us = velocities(m, K)
    T0 = ta.Tb + 0.1 * np.random.default_rng(2).standard_normal(m.n_unique) * ta.mk
    c = adjoint.nusselt_bottom_grad(m, ta.g)
    base = np.dot(c, ta.forward(T0, us))
    free = np.nonzero(m.mask)[0]
    jac = np.zeros(len(free))  # dJ/dT0 by perturbing one free node at a time (J is affine)
    for t, i in enumerate(free):
        T1 = T0.copy()
        T1[i] += 1.0
        jac[t] = np.dot(c, ta.forward(T1, us)) - base
    grad = ta.adjoint(c, us)
    np.testing.assert_allclose(grad[free], jac, rtol=0, atol=1e-10 * np.abs(jac).max())
    assert np.all(grad[m.mask == 0] == 0.0)


def test_adjoint_against_central_differences():
    m = rbc_mesh((2, 2, 3), 4, 1.5)
    K, kappa, dt = 6, 0.02, 0.005
    ta = adjoint.TAdv(m, kappa, dt)
    us = velocities(m, K, amp=0.5, seed=7)
    T0 = ta.Tb.copy()
    J = lambda T: adjoint.nusselt_bottom(m, ta.g, ta.forward(T, us))  # noqa: E731
    grad = ta.adjoint(adjoint.nusselt_bottom_grad(m, ta.g), us)
    rng = np.random.default_rng(11)
    eps = 1e-6
    for _ in range(4):
        d = rng.standard_normal(m.n_unique) * ta.mk
        fd = (J(T0 + eps * d) - J(T0 - eps * d)) / (2 * eps)
        assert abs(fd - np.dot(grad, d)) <= 1e-6 * (abs(fd) + 1e-12), (fd, np.dot(grad, d))


@pytest.mark.parametrize("stretch", [0.0, 1.5])
def test_nusselt_reads_the_bottom_plate_flux(stretch):
    """T = 1 - z + c z (Lz - z)(1 + b x (Lx - x)) lies in the discrete space
    (each element is affine in z with or without the tanh clustering of its
    interfaces), so the GLL quadrature is exact: the bottom plate's mean flux
    gives Nu_b = 1 - c Lz (1 + b Lx^2/6), the top plate's would give
    1 + c Lz (1 + b Lx^2/6). Pins the plate (k = 0 of the bottom elements),
    the sign and the area normalisation."""
    m = rbc_mesh((3, 2, 3), 4, stretch)
    g = rbc.geometry(m)
    x = np.zeros(m.n_unique)
    z = np.zeros(m.n_unique)
    x[m.l2g] = m.X
    z[m.l2g] = m.Z
    Lx, Lz = m.L[0], m.L[2]
    x = np.where(np.isclose(x, Lx), 0.0, x)  # the periodic seam holds one node for x = 0 and x = Lx
    c, b = 0.3, 0.8
    T = 1.0 - z + c * z * (Lz - z) * (1.0 + b * x * (Lx - x))
    expect = 1.0 - c * Lz * (1.0 + b * Lx ** 2 / 6.0)
    assert abs(adjoint.nusselt_bottom(m, g, T) - expect) < 1e-12
    w = adjoint.bottom_weights(m, g)
    assert abs(w.sum() - m.L[0] * m.L[1]) < 1e-12
    assert np.all(w[np.repeat(np.arange(m.E) // (m.nel[0] * m.nel[1]) > 0, (m.N + 1) ** 3)] == 0.0)


def test_transport_replays_the_rbc_temperatures():
    """The frozen-velocity temperature steps are the temperature update of the
    RBC step (Sec. 4.1 Eq. (2)): fed the velocity u^n at the start of every
    step of an oracle RBC run, TAdv.forward reproduces that run's T^1..T^K to
    the solver tolerance. The two are written separately (the lifting enters
    as H_L Tb in one and as (b0/dt) B Tb + kappa A Tb in the other), so a
    dropped term, a wrong BDF/EXT coefficient or a wrong start-up step in
    either breaks the match."""
    m = rbc_mesh((2, 2, 3), 4, 1.5)
    Ra, Pr, dt, K = 2e4, 1.0, 5e-3, 5
    R = rbc.RBC(m, Ra, Pr, dt, tol=1e-13)
    pert = 0.3 * np.random.default_rng(9).standard_normal(m.n_unique)
    s = R.initial_state(pert)
    T0 = s.T.copy()
    us, Ts = [], []
    for _ in range(K):
        us.append([c.copy() for c in s.u])
        s = R.step(s)
        Ts.append(s.T.copy())
    assert max(np.abs(c).max() for c in s.u) > 1e-4  # buoyancy has set the fluid moving
    ta = adjoint.TAdv(m, R.kappa, dt, tol=1e-13)
    for k in range(1, K + 1):
        Tk = ta.forward(T0, us[:k])
        assert np.abs(Tk - Ts[k - 1]).max() < 1e-10, k
    # the velocity matters: replaying with the velocity of the wrong step fails
    shifted = [us[0]] + us[:-1]
    assert np.abs(ta.forward(T0, shifted) - Ts[-1]).max() > 1e-8
