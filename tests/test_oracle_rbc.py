"""Pins of the oracle's Rayleigh-Benard BDF2/EXT2 step (Sec. 4.1, Eqs. (1)-(3);
plates and periodicity of Sec. 4.4): exact steady states, second-order
temporal accuracy on an exact solution, the wall term on an analytic field,
the weak divergence against dense brute force, and the pressure step leaving
a weakly divergence-free velocity (spectrally small in N), the BDF/EXT
coefficients on polynomials, and the onset of convection at the critical
Rayleigh number of linear theory. CPU only."""
import numpy as np
import pytest

import oracle
from oracle import rbc
from bruteforce import gll_numpy


def rbc_mesh(nel=(3, 3, 3), N=5, stretch=2.0):
    return oracle.box_mesh(nel, N, periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), z_stretch=stretch)


def zg(m):
    z = np.zeros(m.n_unique)
    z[m.l2g] = m.Z
    return z


def test_conduction_state_is_a_fixed_point():
    """u = 0, T = 1 - z, p = z - z^2/2 (+c) solve Eqs. (1)-(3) exactly (the
    initial state of Sec. 4.4 without perturbation)."""
    m = rbc_mesh()
    R = rbc.RBC(m, 1e8, 0.7, 1e-3, tol=1e-13)
    s = R.initial_state()
    z = zg(m)
    pex = z - z * z / 2
    pex -= pex.mean()
    for _ in range(3):
        s = R.step(s)
        assert np.abs(s.T - (1.0 - z)).max() < 1e-13
        assert max(np.abs(c).max() for c in s.u) < 1e-13
        assert np.abs(s.p - pex).max() < 1e-11


def test_second_order_in_time_on_diffusing_profile():
    """T = 1 - z + a exp(-kappa pi^2 t) sin(pi z), u = 0 solves the system
    (buoyancy balanced by a hydrostatic pressure). BDF2/EXT2 error ~ dt^2."""
    Ra, Pr, a, tend = 100.0, 1.0, 0.3, 0.24
    kappa = 1.0 / np.sqrt(Ra * Pr)
    m = rbc_mesh((2, 2, 4), 8, stretch=0.0)
    z = zg(m)
    errs = []
    for nsteps in (6, 12, 24):
        dt = tend / nsteps
        R = rbc.RBC(m, Ra, Pr, dt, tol=1e-13)
        s = R.initial_state(a * np.sin(np.pi * z))
        for _ in range(nsteps):
            s = R.step(s)
        exact = 1.0 - z + a * np.exp(-kappa * np.pi ** 2 * tend) * np.sin(np.pi * z)
        errs.append(np.abs(s.T - exact).max())
        assert max(np.abs(c).max() for c in s.u) < 1e-9
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, errs


def test_wall_term_on_analytic_field():
    """u = (x z, 0, 0) has curl curl u = (0, 0, 1): the wall term is
    nu * (-1 on z = 0, +1 on z = Lz) times the surface quadrature weights."""
    L = (1.0, 1.5, 0.8)
    nel, N, nu = (3, 2, 2), 4, 0.37
    m = oracle.box_mesh(nel, N, L, periodic=(0, 0, 0), dirichlet=(0, 0, 0, 0, 1, 1))
    g = rbc.geometry(m)
    u = [m.X * m.Z, np.zeros(m.n_local), np.zeros(m.n_local)]
    W = rbc.wall_term(m, g, u, nu)
    hx, hy = L[0] / nel[0], L[1] / nel[1]
    _, rho, _ = gll_numpy(N)
    n = N + 1
    ref = np.zeros(m.n_local)
    e = np.arange(m.E)
    ez = e // (nel[0] * nel[1])
    for el in e:
        for k, sgn, hit in ((0, -1.0, ez[el] == 0), (N, 1.0, ez[el] == nel[2] - 1)):
            if not hit:
                continue
            for j in range(n):
                for i in range(n):
                    ref[el * n ** 3 + i + n * j + n * n * k] += sgn * nu * rho[i] * rho[j] * hx * hy / 4
    np.testing.assert_allclose(W, oracle.gather_sum(m, ref), rtol=0, atol=1e-12)


def test_weak_divergence_matches_dense():
    from bruteforce import element_matrices  # noqa: F401 (same construction)
    m = oracle.box_mesh((2, 1, 2), 4, deform_amp=0.05, kappa=np.array([[1.0, 2, 1], [2, 1, 1], [1, 1, 2]]),
                        phi=np.array([0.3, 1.7, 4.1]))
    g = rbc.geometry(m)
    rng = np.random.default_rng(9)
    f = [rng.standard_normal(m.n_local) for _ in range(3)]
    got = rbc.weak_div(m, g, f)
    _, rho, D = gll_numpy(m.N)
    n = m.N + 1
    I = np.eye(n)
    grads = (np.kron(I, np.kron(I, D)), np.kron(I, np.kron(D, I)), np.kron(D, np.kron(I, I)))
    ref = np.zeros(m.n_local)
    for el in range(m.E):
        sl = slice(el * n ** 3, (el + 1) * n ** 3)
        Jm = np.zeros((n ** 3, 3, 3))
        for c, xc in enumerate((m.X[sl], m.Y[sl], m.Z[sl])):
            for a in range(3):
                Jm[:, c, a] = grads[a] @ xc
        Rm = np.linalg.inv(Jm)
        w = np.kron(np.kron(rho, rho), rho) * np.linalg.det(Jm)
        for c in range(3):
            Gc = sum(Rm[:, a, c][:, None] * grads[a] for a in range(3))  # d phi / dx_c at nodes
            ref[sl] += Gc.T @ (w * f[c][sl])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_gradient_exact_for_polynomials():
    m = oracle.box_mesh((2, 3, 2), 5, L=(1.0, 2.0, 0.7), z_stretch=1.3)
    g = rbc.geometry(m)
    f = m.X ** 2 * m.Y + m.Z ** 3 - 2.0 * m.X * m.Z
    gr = rbc.grad(m, g, f)
    np.testing.assert_allclose(gr[0], 2 * m.X * m.Y - 2 * m.Z, atol=1e-11)
    np.testing.assert_allclose(gr[1], m.X ** 2, atol=1e-11)
    np.testing.assert_allclose(gr[2], 3 * m.Z ** 2 - 2 * m.X, atol=1e-11)


def test_pressure_step_makes_velocity_weakly_divergence_free():
    """After steps from a smooth perturbation, the weak divergence of the new
    velocity, relative to its size, decays spectrally with the order N and is
    far below that of the same steps with the pressure solve removed (a
    mistake planted in the oracle: the Neumann solve returns zero)."""
    ratios, ablated = [], []
    for N in (3, 5, 7):
        m = rbc_mesh((3, 3, 3), N)
        xg, yg, zgv = np.zeros(m.n_unique), np.zeros(m.n_unique), np.zeros(m.n_unique)
        xg[m.l2g], yg[m.l2g], zgv[m.l2g] = m.X, m.Y, m.Z
        pert = 0.1 * np.sin(np.pi * zgv) * np.cos(2 * np.pi * xg) * np.cos(2 * np.pi * yg)

        def run(no_pressure):
            R = rbc.RBC(m, 1e5, 0.7, 2e-2, tol=1e-13)
            orig = rbc._pcg_neumann
            if no_pressure:
                def zero(m_, b, tol, maxit, x0=None):
                    r = orig(m_, b, tol, maxit, x0=x0)
                    r.x = np.zeros_like(r.x)
                    return r
                rbc._pcg_neumann = zero
            try:
                s = R.initial_state(pert)
                for _ in range(3):
                    s = R.step(s)
            finally:
                rbc._pcg_neumann = orig
            uL = [oracle.scatter(m, c) for c in s.u]
            wd = oracle.gather_sum(m, rbc.weak_div(m, R.geo, uL))
            unorm = np.sqrt(sum(oracle.gather_sum(m, m.B * uL[c] * uL[c]).sum() for c in range(3)))
            return np.linalg.norm(wd) / unorm

        ratios.append(run(False))
        ablated.append(run(True))
    assert ratios[0] > ratios[1] > ratios[2], ratios
    assert ratios[2] < ratios[0] / 10, ratios
    for r, a in zip(ratios, ablated):
        assert r < a / 10, (ratios, ablated)


def test_bdf_ext_coefficients_are_exact_on_polynomials():
    """The time-stepping coefficients (b0, b1, b2, a1, a2) of the step from
    level n: (b0 f^{n+1} - b1 f^n - b2 f^{n-1}) / dt is exact for f' at
    t^{n+1} on polynomials of the scheme's order (quadratics for BDF2, lines
    for the BDF1 first step) and a1 f^n + a2 f^{n-1} extrapolates f^{n+1}
    exactly on lines (EXT2) and constants (EXT1). Taylor tables of the
    textbook schemes, checked on every monomial."""
    dt = 0.37
    for step, order in ((0, 1), (1, 2), (5, 2)):
        b0, b1, b2, a1, a2 = rbc.coefficients(step)
        for p in range(order + 1):
            f = lambda t: (t / dt) ** p  # noqa: E731
            df = p * (1.0 / dt) ** p * dt ** (p - 1) if p else 0.0  # f'(dt) for f = (t/dt)^p
            bdf = (b0 * f(dt) - b1 * f(0.0) - b2 * f(-dt)) / dt
            assert abs(bdf - df) < 1e-14 * max(1.0, abs(df)), (step, p)
        for p in range(order):
            f = lambda t: (t / dt) ** p  # noqa: E731
            assert abs(a1 * f(0.0) + a2 * f(-dt) - f(dt)) < 1e-14, (step, p)
        # and they are not exact one order higher (the scheme is of that order, no more)
        f = lambda t: (t / dt) ** (order + 1)  # noqa: E731
        assert abs((b0 * f(dt) - b1 * f(0.0) - b2 * f(-dt)) / dt - (order + 1) / dt) > 1e-3


def _onset_growth_rate(Ra, kc=3.117, dt=0.1, steps=160):
    """Exponential growth rate of |w| for a perturbation T' = 1e-4 sin(pi z)
    cos(kc x) in a box holding one wavelength, rigid isothermal plates,
    Pr = 1 (fit over the second half of the run)."""
    Lx = 2.0 * np.pi / kc
    m = oracle.box_mesh((4, 1, 4), 5, L=(Lx, 0.5, 1.0), periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1))
    R = rbc.RBC(m, Ra, 1.0, dt, tol=1e-11)
    x, z = np.zeros(m.n_unique), np.zeros(m.n_unique)
    x[m.l2g], z[m.l2g] = m.X, m.Z
    s = R.initial_state(1e-4 * np.sin(np.pi * z) * np.cos(kc * x))
    amp = []
    for _ in range(steps):
        s = R.step(s)
        amp.append(np.linalg.norm(s.u[2]))
    t = dt * np.arange(1, steps + 1)
    h = steps // 2
    return np.polyfit(t[h:], np.log(np.array(amp[h:])), 1)[0]


def test_onset_of_convection_at_the_critical_rayleigh_number():
    """Linear stability of the Boussinesq equations (Sec. 4.1, Eqs. (1)-(3))
    between rigid isothermal plates (Sec. 4.4): the conduction state loses
    stability at Ra_c = 1707.76 with critical wavenumber k_c = 3.117
    (Chandrasekhar 1961). The critical mode decays at Ra = 1650 and grows at
    1770, and the zero of the growth rate (secant) lies within 1 % of Ra_c.
    A wrong sign or scale of buoyancy, viscosity or diffusivity, or slip
    walls, moves or removes the onset."""
    s_lo, s_hi = _onset_growth_rate(1650.0), _onset_growth_rate(1770.0)
    assert s_lo < 0.0 < s_hi, (s_lo, s_hi)
    ra0 = 1650.0 + 120.0 * (-s_lo) / (s_hi - s_lo)
    assert abs(ra0 / 1707.76 - 1.0) < 0.01, ra0


def test_extrapolated_initial_guesses_change_only_the_iterations():
    """Starting every solve of a step from 2 x^n - x^{n-1} (the option for the
    RBC solves) leaves the fields of the step the same up to the solver
    tolerance, steps from the conduction state stay at it, and from the
    second step on the Helmholtz solves need fewer iterations."""
    m = rbc_mesh((2, 2, 3), 4, 1.5)
    pert = 0.2 * np.random.default_rng(5).standard_normal(m.n_unique)
    runs = {}
    for ex in (False, True):
        R = rbc.RBC(m, 2e4, 1.0, 5e-3, tol=1e-11, extrapolate=ex)
        s = R.initial_state(pert)
        hist = []
        for _ in range(5):
            s = R.step(s)
            hist.append(s.iters)
        runs[ex] = (s, hist)
    (s0, h0), (s1, h1) = runs[False], runs[True]
    assert np.abs(s1.T - s0.T).max() < 1e-9
    assert max(np.abs(a - b).max() for a, b in zip(s1.u, s0.u)) < 1e-9
    assert np.abs(s1.p - s0.p).max() < 1e-7 * max(1.0, np.abs(s0.p).max())
    assert h1[0] == h0[0]  # the first step has no history to extrapolate from
    later0 = sum(h["T"] + sum(h["u"]) for h in h0[2:])
    later1 = sum(h["T"] + sum(h["u"]) for h in h1[2:])
    assert later1 < later0, (h0, h1)
    R = rbc.RBC(m, 1e8, 0.7, 1e-3, tol=1e-13, extrapolate=True)  # conduction stays a fixed point
    s = R.initial_state()
    z = zg(m)
    for _ in range(3):
        s = R.step(s)
        assert np.abs(s.T - (1.0 - z)).max() < 1e-13


def test_third_order_guesses_change_only_the_iterations():
    """extrapolate = 2 (temperature and velocity from 3x^n - 3x^{n-1} +
    x^{n-2} once three levels exist, pressure from 2p^n - p^{n-1}) leaves the
    fields the same up to the solver tolerance, gives the first two steps the
    iterations of the second-order option, and needs no more Helmholtz
    iterations than it afterwards; conduction stays a fixed point."""
    m = rbc_mesh((2, 2, 3), 4, 1.5)
    pert = 0.2 * np.random.default_rng(5).standard_normal(m.n_unique)
    runs = {}
    for ex in (1, 2):
        R = rbc.RBC(m, 2e4, 1.0, 5e-3, tol=1e-11, extrapolate=ex)
        s = R.initial_state(pert)
        hist = []
        for _ in range(8):
            s = R.step(s)
            hist.append(s.iters)
        runs[ex] = (s, hist)
    (s1, h1), (s2, h2) = runs[1], runs[2]
    assert np.abs(s2.T - s1.T).max() < 1e-9
    assert max(np.abs(a - b).max() for a, b in zip(s2.u, s1.u)) < 1e-9
    assert np.abs(s2.p - s1.p).max() < 1e-7 * max(1.0, np.abs(s1.p).max())
    assert h2[:2] == h1[:2]  # third order needs three earlier levels
    later1 = sum(h["T"] + sum(h["u"]) for h in h1[2:])
    later2 = sum(h["T"] + sum(h["u"]) for h in h2[2:])
    assert later2 < later1, (h1, h2)
    R = rbc.RBC(m, 1e8, 0.7, 1e-3, tol=1e-13, extrapolate=2)
    s = R.initial_state()
    z = zg(m)
    for _ in range(4):
        s = R.step(s)
        assert np.abs(s.T - (1.0 - z)).max() < 1e-13
