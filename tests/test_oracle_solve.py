"""Pins of the oracle's preconditioned CG solve (Sec. 2.2: the pressure
Poisson solve, preconditioned) and of the grid-point convention of the
paper's Table "Details of the simulations with Gamma = 4". CPU only."""
import os

import numpy as np
import pytest

import oracle
from bruteforce import dense_global
from workloads import BoxWorkload, POISSON_4

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gridpoint_convention_matches_paper_table():
    """Grid points = N_e * p^3, as printed in the paper's simulation table."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "sim_details_gridpoints.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 8
    for ra, nx, ny, nz, p, printed, unit in rows:
        w = BoxWorkload("t", (int(nx), int(ny), int(nz)), N=int(p))
        scale = 1e6 if unit == "million" else 1e9
        val = float(printed) * scale
        digits = len(printed.replace(".", "").lstrip("0"))
        # the printed figure is the count truncated/rounded to its printed digits
        assert abs(w.dofs - val) <= 10 ** (np.floor(np.log10(val)) - digits + 1), (ra, w.dofs, val)


@pytest.mark.parametrize("nel,N,deform,h1,h2", [((2, 2, 2), 3, 0.05, 1.0, 0.0), ((2, 1, 2), 4, 0.0, 1.0, 0.0),
                                               ((2, 2, 1), 4, 0.05, 0.3, 20.0), ((1, 1, 1), 6, 0.04, 1.0, 0.0)])
def test_pcg_matches_dense_direct_solve(nel, N, deform, h1, h2):
    kap = np.array([[1.0, 2.0, 1.0], [2.0, 1.0, 1.0], [1.0, 1.0, 2.0]])
    m = oracle.box_mesh(nel, N, deform_amp=deform, kappa=kap, phi=np.array([0.3, 1.7, 4.1]))
    Ag, _, _ = dense_global(m, h1, h2)
    free = m.mask == 1
    b = np.random.default_rng(7).standard_normal(m.n_unique) * m.mask
    x_ref = np.zeros(m.n_unique)
    x_ref[free] = np.linalg.solve(Ag[np.ix_(free, free)], b[free])
    res = oracle.pcg(m, b, h1, h2, tol=1e-14, maxit=2000)
    assert res.converged
    np.testing.assert_allclose(res.x, x_ref, rtol=0, atol=1e-12 * np.abs(x_ref).max())
    # unpreconditioned CG reaches the same solution
    res0 = oracle.pcg(m, b, h1, h2, tol=1e-14, maxit=4000, precond="none")
    np.testing.assert_allclose(res0.x, x_ref, rtol=0, atol=1e-11 * np.abs(x_ref).max())


def test_spectral_convergence_manufactured_poisson():
    """||u_h - u||_inf for -lap u = 3 pi^2 u, u = sin sin sin on 4^3 elements
    decays exponentially in N (the spec spectral-convergence check)."""
    errs = {}
    for N in range(2, 11):
        m = oracle.box_mesh((4, 4, 4), N)
        res = oracle.pcg(m, oracle.poisson_rhs(m), tol=1e-13, maxit=3000)
        assert res.converged
        u = oracle.manufactured_u(m)
        errs[N] = np.abs(oracle.scatter(m, res.x) - u).max()
    Ns = [n for n in sorted(errs) if n <= 8]  # from N = 9 on the error is at round-off
    for a, b in zip(Ns[:-1], Ns[1:]):
        assert errs[b] < errs[a] * 0.2, errs  # rapidly decreasing
    assert errs[9] < 1e-13 and errs[10] < 1e-13
    # exponential: log-error roughly linear in N with slope < -2 per order
    slope = np.polyfit(Ns, np.log(np.array([errs[n] for n in Ns])), 1)[0]
    assert slope < -2.0, (slope, errs)


def test_poisson_4_workload_reaches_tolerance():
    m = oracle.mesh_from_workload(POISSON_4)
    res = oracle.pcg(m, oracle.poisson_rhs(m), tol=1e-10, maxit=1000)
    assert res.converged and res.rel_residual <= 1e-10
    err = np.abs(oracle.scatter(m, res.x) - oracle.manufactured_u(m)).max()
    assert err < 1e-5
    # residual history decreases overall; Jacobi PCG on this mesh needs < 200 iterations
    assert res.iterations < 200


def test_pcg_zero_rhs_returns_zero():
    m = oracle.box_mesh((1, 1, 1), 3)
    res = oracle.pcg(m, np.zeros(m.n_unique))
    assert res.iterations == 0 and res.converged and not res.x.any()


def test_pcg_initial_guess_solves_the_same_system():
    """From an initial guess x0 the oracle's PCG starts at r0 = b - A x0 and
    keeps the stopping test ||r|| <= tol ||b||: it reaches the solution of the
    zero-start solve (a sign error in r0 would converge elsewhere), in fewer
    iterations from a nearby guess, and returns the guess itself, with no
    iteration, when the guess already meets the tolerance."""
    m = oracle.box_mesh((2, 2, 2), 4, deform_amp=0.05, kappa=np.full(9, 1.0), phi=np.array([0.1, 0.2, 0.3]))
    rng = np.random.default_rng(3)
    b = rng.standard_normal(m.n_unique) * m.mask
    ref = oracle.pcg(m, b, 1.0, 0.3, tol=1e-13, maxit=2000)
    far = oracle.pcg(m, b, 1.0, 0.3, tol=1e-13, maxit=2000, x0=rng.standard_normal(m.n_unique) * m.mask)
    assert far.converged and np.abs(far.x - ref.x).max() < 1e-11 * np.abs(ref.x).max()
    near_guess = ref.x + 1e-6 * rng.standard_normal(m.n_unique) * m.mask
    near = oracle.pcg(m, b, 1.0, 0.3, tol=1e-10, maxit=2000, x0=near_guess)
    zero = oracle.pcg(m, b, 1.0, 0.3, tol=1e-10, maxit=2000)
    assert near.converged and near.iterations < zero.iterations
    done = oracle.pcg(m, b, 1.0, 0.3, tol=1e-10, maxit=2000, x0=ref.x)
    assert done.iterations == 0 and np.array_equal(done.x, ref.x)
