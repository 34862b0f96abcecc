"""Pins of the oracle's p-multigrid preconditioner (Sec. 2.2: p-multigrid with
4th-kind Chebyshev-accelerated smoothing): interpolation exactness, R = P^T,
the 4th-kind Chebyshev error bound 1/(2k+1) (Lottes 2022), V-cycle symmetry,
and the preconditioned flexible CG against a dense direct solve, for the
Poisson and the Helmholtz operator. CPU only."""
import numpy as np
import numpy.polynomial.legendre as npl
import pytest

import oracle
from oracle import pmg
from bruteforce import dense_global

KAPPA = np.array([[1.0, 2.0, 1.0], [2.0, 1.0, 1.0], [1.0, 1.0, 2.0]])
PHI = np.array([0.3, 1.7, 4.1])


def test_lagrange_matrix_reproduces_polynomials():
    for nc, nf in ((3, 7), (1, 3), (2, 9)):
        xc, _, _ = oracle.gll(nc)
        xf, _, _ = oracle.gll(nf)
        J = pmg.lagrange_matrix(xc, xf)
        np.testing.assert_allclose(J.sum(axis=1), 1.0, atol=1e-14)
        for d in range(nc + 1):
            np.testing.assert_allclose(J @ xc ** d, xf ** d, atol=1e-13)
        # and not beyond degree nc
        assert np.abs(J @ xc ** (nc + 1) - xf ** (nc + 1)).max() > 1e-6


def box(nel, deform=0.0, L=(1.0, 1.0, 1.0)):
    return dict(nel=nel, L=L, deform_amp=deform, kappa=KAPPA, phi=PHI)


def test_prolongation_exact_on_coarse_polynomials():
    pm = pmg.PMG(box((2, 3, 2), L=(1.0, 1.5, 0.8)), orders=(7, 3, 1))
    for l in range(2):
        mf, mc = pm.levels[l].m, pm.levels[l + 1].m
        f = lambda X, Y, Z: X ** 2 * Y - 0.5 * Z ** 3 * X + Y * Z  # noqa: E731 (degree <= 3 per direction)
        if mc.N == 1:
            f = lambda X, Y, Z: X * Y * Z + 2 * X - Y  # noqa: E731
        uc = np.zeros(mc.n_unique)
        uc[mc.l2g] = f(mc.X, mc.Y, mc.Z)
        uf = np.zeros(mf.n_unique)
        uf[mf.l2g] = f(mf.X, mf.Y, mf.Z)
        np.testing.assert_allclose(pm.prolong(l, uc), uf, atol=1e-12)


def test_restriction_is_the_transpose():
    pm = pmg.PMG(box((2, 2, 3), 0.05), orders=(5, 2, 1))
    rng = np.random.default_rng(3)
    for l in range(2):
        mf, mc = pm.levels[l].m, pm.levels[l + 1].m
        a, b = rng.standard_normal(mc.n_unique), rng.standard_normal(mf.n_unique)
        assert abs(np.dot(pm.prolong(l, a), b) - np.dot(a, pm.restrict(l, b))) < 1e-12 * np.sqrt(mf.n_unique)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_chebyshev_fourth_kind_error_bound(k):
    """The 4th-kind Chebyshev smoother's error polynomial p_k satisfies
    max_t |p_k(t)| sqrt(t/lam) = 1/(2k+1) on (0, lam] (equioscillation)."""
    m = oracle.box_mesh((2, 2, 2), 3, deform_amp=0.05, kappa=KAPPA, phi=PHI)
    pm = pmg.PMG(dict(nel=(2, 2, 2), deform_amp=0.05, kappa=KAPPA, phi=PHI), orders=(3, 1), degree=k)
    lev = pm.levels[0]
    Ag, _, _ = dense_global(m)
    free = m.mask == 1
    A = Ag[np.ix_(free, free)]
    dvec = np.diag(A)
    lam_true = np.linalg.eigvalsh(A / np.sqrt(np.outer(dvec, dvec))).max()
    lev.lam = lam_true  # exact lambda_max: the bound is then attained
    t, V = np.linalg.eigh(A / np.sqrt(np.outer(dvec, dvec)))
    worst = 0.0
    for i in range(len(t)):
        v = np.zeros(m.n_unique)
        v[free] = V[:, i] / np.sqrt(dvec)  # eigenvector of D^{-1} A
        e = v - pm.smooth(0, pm.A(0, v))   # error propagation E = I - S A
        p = np.dot(e[free], dvec * v[free]) / np.dot(v[free], dvec * v[free])
        worst = max(worst, abs(p) * np.sqrt(t[i] / lam_true))
    assert worst <= (1.0 + 1e-9) / (2 * k + 1)
    assert worst >= 0.9 / (2 * k + 1)


@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.3, 25.0)])
def test_vcycle_is_symmetric_with_exact_coarse_solve(h1, h2):
    pm = pmg.PMG(box((2, 2, 2), 0.05), orders=(5, 2, 1), h1=h1, h2=h2, coarse_tol=1e-14)
    rng = np.random.default_rng(5)
    mk = pm.levels[0].mk
    a, b = rng.standard_normal(len(mk)) * mk, rng.standard_normal(len(mk)) * mk
    x, y = np.dot(pm.vcycle(a), b), np.dot(a, pm.vcycle(b))
    assert abs(x - y) <= 1e-10 * abs(x)


def test_fcg_matches_direct_solve_and_beats_jacobi():
    bx = box((3, 2, 2), 0.05)
    pm = pmg.PMG(bx, orders=(6, 3, 1))
    m = pm.levels[0].m
    Ag, _, _ = dense_global(m)
    free = m.mask == 1
    b = np.random.default_rng(8).standard_normal(m.n_unique) * m.mask
    x_ref = np.zeros(m.n_unique)
    x_ref[free] = np.linalg.solve(Ag[np.ix_(free, free)], b[free])
    res = pmg.fcg(pm, b, tol=1e-12, maxit=100)
    assert res.converged
    np.testing.assert_allclose(res.x, x_ref, rtol=0, atol=1e-10 * np.abs(x_ref).max())
    jac = oracle.pcg(m, b, tol=1e-12, maxit=2000)
    assert res.iterations * 4 < jac.iterations, (res.iterations, jac.iterations)


def test_fcg_helmholtz_matches_direct_solve():
    """h1 A + h2 B (the implicit diffusion operators of the time step): the
    hierarchy re-discretises both terms on every level, and the flexible CG
    reaches the dense direct solution of the masked Helmholtz system."""
    bx = box((3, 2, 2), 0.05)
    h1, h2 = 0.02, 400.0  # diffusion-to-mass ratio of the order of a time step's
    pm = pmg.PMG(bx, orders=(6, 3, 1), h1=h1, h2=h2)
    m = pm.levels[0].m
    Hg, _, _ = dense_global(m, h1, h2)
    free = m.mask == 1
    b = np.random.default_rng(9).standard_normal(m.n_unique) * m.mask
    x_ref = np.zeros(m.n_unique)
    x_ref[free] = np.linalg.solve(Hg[np.ix_(free, free)], b[free])
    res = pmg.fcg(pm, b, tol=1e-12, maxit=100)
    assert res.converged
    np.testing.assert_allclose(res.x, x_ref, rtol=0, atol=1e-10 * np.abs(x_ref).max())
    jac = oracle.pcg(m, b, h1, h2, tol=1e-12, maxit=2000)
    assert res.iterations <= jac.iterations, (res.iterations, jac.iterations)


@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.3, 25.0)])
def test_power_iteration_converges_to_lambda_max(h1, h2):
    """The smoother's eigenvalue bound: the power iteration on D^{-1} A
    (started from the checkerboard vector) tends to the largest eigenvalue
    of the dense D^{-1/2} A D^{-1/2}; within 1 % after the default 20
    iterations, which the 1.1 safety factor covers."""
    m = oracle.box_mesh((2, 2, 2), 4, deform_amp=0.05, kappa=KAPPA, phi=PHI)
    Ag, _, _ = dense_global(m, h1=h1, h2=h2)
    free = m.mask == 1
    A = Ag[np.ix_(free, free)]
    d = np.diag(A)
    lam = np.linalg.eigvalsh(A / np.sqrt(np.outer(d, d))).max()
    boxd = dict(nel=(2, 2, 2), deform_amp=0.05, kappa=KAPPA, phi=PHI)
    long = pmg.PMG(boxd, orders=(4, 1), h1=h1, h2=h2, power_its=400, safety=1.0).levels[0].lam
    assert abs(long / lam - 1.0) < 1e-6
    short = pmg.PMG(boxd, orders=(4, 1), h1=h1, h2=h2, safety=1.0).levels[0].lam
    assert abs(short / lam - 1.0) < 1e-2
    assert pmg.PMG(boxd, orders=(4, 1), h1=h1, h2=h2).levels[0].lam == pytest.approx(1.1 * short, rel=1e-15)
