"""Pins of the oracle's mesh, geometry, local operator and direct-stiffness
summation (Sec. 2.2: matrix-free tensor contractions carried to deformed
elements by the chain rule) against closed forms, invariants and dense brute
force. CPU only."""
import dataclasses

import numpy as np
import pytest

import oracle
from bruteforce import dense_global, element_matrices, gll_numpy, unique_classes

KAPPA = np.array([[1.0, 2.0, 1.0], [2.0, 1.0, 1.0], [1.0, 1.0, 2.0]])
PHI = np.array([0.3, 1.7, 4.1])


def small_mesh(nel=(2, 2, 2), N=4, deform=0.0, periodic=(0, 0, 0), dirichlet=(1,) * 6, stretch=0.0, L=(1.0, 1.0, 1.0)):
    return oracle.box_mesh(nel, N, L, periodic, dirichlet, stretch, deform, KAPPA, PHI)


# ---------------------------------------------------------------- index maps
@pytest.mark.parametrize("nel,periodic", [((2, 2, 2), (0, 0, 0)), ((3, 2, 1), (0, 0, 0)),
                                          ((2, 3, 2), (1, 1, 0)), ((3, 3, 3), (1, 1, 1)),
                                          ((1, 1, 1), (0, 0, 0))])
def test_l2g_classes_equal_coordinate_classes(nel, periodic):
    m = small_mesh(nel, 3, periodic=periodic)
    cls = unique_classes((m.X, m.Y, m.Z), m.L, periodic)
    # the same partition of local nodes: a bijection between class ids
    pairs = np.unique(np.stack([cls, m.l2g], axis=1), axis=0)
    assert len(pairs) == len(np.unique(cls)) == len(np.unique(m.l2g)) == m.n_unique


def test_l2g_numbering_is_lexicographic_in_z_y_x():
    m = small_mesh((3, 2, 2), 3)
    order = np.lexsort((m.X, m.Y, m.Z))  # z slowest, x fastest
    ranks = np.empty(m.n_local, dtype=np.int64)
    uniq_sorted = np.unique(np.stack([np.round(m.Z * 1e9), np.round(m.Y * 1e9), np.round(m.X * 1e9)], 1)[order],
                            axis=0, return_inverse=True)[1].ravel()
    ranks[order] = uniq_sorted
    np.testing.assert_array_equal(ranks, m.l2g)


def test_multiplicities_box():
    nel = 3
    m = small_mesh((nel,) * 3, 2)
    mult = m.mult
    vals, counts = np.unique(mult, return_counts=True)
    got = dict(zip(vals.astype(int), counts))
    # unique lattice nodes with 1 (element interior or boundary-only), 2 (shared face),
    # 4 (shared edge) and 8 (shared vertex) copies in an nel^3 box with N = 2
    assert got[8] == (nel - 1) ** 3
    assert got[4] == 3 * (nel - 1) ** 2 * (2 + nel * 1)
    assert sum(got.values()) == m.n_unique
    assert float(mult.sum()) == m.n_local


def test_qqt_twice_is_mult_times_qqt():
    m = small_mesh((2, 2, 2), 3, deform=0.05)
    v = np.random.default_rng(5).standard_normal(m.n_local)
    once = oracle.qqt(m, v)
    twice = oracle.qqt(m, once)
    np.testing.assert_allclose(twice, oracle.scatter(m, m.mult) * once, rtol=1e-14)


def test_mask_marks_dirichlet_faces():
    m = small_mesh((2, 2, 2), 3, periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1))
    zg = np.zeros(m.n_unique)
    zg[m.l2g] = m.Z
    np.testing.assert_array_equal(m.mask == 0, np.isclose(zg, 0.0) | np.isclose(zg, 1.0))


# ---------------------------------------------------------------- geometry
def test_affine_geometric_factors_closed_form():
    L = (1.0, 2.0, 0.5)
    nel = (2, 3, 1)
    N = 5
    m = small_mesh(nel, N, L=L)
    h = [L[d] / nel[d] for d in range(3)]
    _, rho, _ = oracle.gll(N)
    w = np.kron(np.kron(rho, rho), rho)
    w = np.tile(w, m.E)
    vol = h[0] * h[1] * h[2] / 8.0
    np.testing.assert_allclose(m.B, w * vol, rtol=1e-13)
    diag = {0: 0, 3: 1, 5: 2}
    for f in range(6):
        if f in diag:
            np.testing.assert_allclose(m.G[f], w * vol * (2.0 / h[diag[f]]) ** 2, rtol=1e-12)
        else:
            np.testing.assert_allclose(m.G[f], 0.0, atol=1e-13)


def test_polynomial_map_geometry_matches_analytic_jacobian():
    """A map polynomial of degree <= N in each reference direction is
    interpolated exactly, so the D-derivative equals the analytic Jacobian."""
    N = 4
    base = small_mesh((2, 2, 2), N)
    x0, y0, z0 = base.X, base.Y, base.Z
    X = x0 + 0.1 * y0 * y0 * z0
    Y = y0 + 0.05 * x0 * z0
    Z = z0 + 0.08 * x0 * x0 - 0.03 * y0
    m = oracle.box_mesh((2, 2, 2), N, coords=(X, Y, Z))
    # analytic dX/dx0 (global), times the affine reference Jacobian h/2
    h = 0.5
    Jg = np.zeros((m.n_local, 3, 3))
    Jg[:, 0] = np.stack([np.ones_like(x0), 0.2 * y0 * z0, 0.1 * y0 * y0], 1)
    Jg[:, 1] = np.stack([0.05 * z0, np.ones_like(x0), 0.05 * x0], 1)
    Jg[:, 2] = np.stack([0.16 * x0, -0.03 * np.ones_like(x0), np.ones_like(x0)], 1)
    Jr = Jg * (h / 2.0)
    det = np.linalg.det(Jr)
    R = np.linalg.inv(Jr)
    _, rho, _ = oracle.gll(N)
    w = np.tile(np.kron(np.kron(rho, rho), rho), m.E) * det
    np.testing.assert_allclose(m.B, w, rtol=1e-12)
    pa, pb = [0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]
    for f in range(6):
        ref = w * np.einsum("qc,qc->q", R[:, pa[f], :], R[:, pb[f], :])
        np.testing.assert_allclose(m.G[f], ref, rtol=1e-10, atol=1e-14)


def test_mass_sums_to_volume():
    m = small_mesh((3, 2, 2), 6, deform=0.1)
    assert abs(m.B.sum() - 1.0) < 1e-6  # GLL quadrature of det J (spectrally accurate)
    m = small_mesh((3, 2, 2), 6, stretch=2.0)
    assert abs(m.B.sum() - 1.0) < 1e-13  # straight-sided: exact


def test_tanh_interfaces():
    """Element interfaces follow z_k = 1/2 [1 + tanh(s(2k/n - 1))/tanh(s)]."""
    s, nz = 2.0, 4
    m = small_mesh((1, 1, nz), 2, stretch=s)
    n = 3
    zs = [m.Z[e * n ** 3] for e in range(nz)] + [m.Z[(nz - 1) * n ** 3 + n * n * (n - 1)]]
    ref = 0.5 * (1.0 + np.tanh(s * (2.0 * np.arange(nz + 1) / nz - 1.0)) / np.tanh(s))
    np.testing.assert_allclose(zs, ref, rtol=1e-15, atol=1e-16)


# ---------------------------------------------------------------- operator
CASES = [((1, 1, 1), 1, 0.0), ((1, 1, 1), 3, 0.04), ((2, 1, 1), 4, 0.05), ((2, 2, 2), 2, 0.05),
         ((2, 2, 2), 5, 0.0), ((1, 2, 1), 8, 0.05), ((2, 2, 2), 3, 0.05)]


@pytest.mark.parametrize("nel,N,deform", CASES)
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.7, 3.5)])
def test_ax_matches_dense_bruteforce(nel, N, deform, h1, h2):
    m = small_mesh(nel, N, deform=deform)
    Ag, AL, Q = dense_global(m, h1, h2)
    u = np.random.default_rng(1).uniform(-1, 1, m.n_local)
    scale = np.abs(AL).max() * np.abs(u).max() * (N + 1) ** 3
    np.testing.assert_allclose(oracle.ax_local(m, u, h1, h2), AL @ u, rtol=0, atol=1e-14 * scale)
    ug = np.random.default_rng(2).uniform(-1, 1, m.n_unique)
    mk = m.mask.astype(float)
    ref = mk * (Ag @ (mk * ug))
    np.testing.assert_allclose(oracle.apply_assembled(m, ug, h1, h2), ref, rtol=0, atol=1e-14 * scale)
    # Jacobi diagonal
    np.testing.assert_allclose(oracle.diag_assembled(m, h1, h2), np.diag(Ag), rtol=1e-12,
                               atol=1e-14 * np.abs(Ag).max())


def test_bruteforce_uses_independent_basis():
    for N in (2, 5, 9):
        xi, rho, D = oracle.gll(N)
        xn, rn, Dn = gll_numpy(N)
        np.testing.assert_allclose(xi, xn, atol=1e-14)
        np.testing.assert_allclose(D, Dn, atol=1e-10 * N * N)


def test_symmetry_and_null_space():
    m = small_mesh((2, 2, 2), 5, deform=0.05)
    rng = np.random.default_rng(3)
    u, v = rng.standard_normal(m.n_local), rng.standard_normal(m.n_local)
    Au, Av = oracle.ax_local(m, u), oracle.ax_local(m, v)
    assert abs(v @ Au - u @ Av) <= 1e-14 * np.abs(v) @ np.abs(Au)
    one = np.ones(m.n_local)
    A1 = oracle.ax_local(m, one)
    assert np.abs(A1).max() < 1e-12 * np.abs(Au).max()
    # assembled Neumann operator (no mask) annihilates constants as well
    Ag1 = oracle.gather_sum(m, oracle.ax_local(m, oracle.scatter(m, np.ones(m.n_unique))))
    assert np.abs(Ag1).max() < 1e-12 * np.abs(Au).max()
    # SPD on the masked space
    ug = rng.standard_normal(m.n_unique) * m.mask
    assert ug @ oracle.apply_assembled(m, ug) > 0.0


def test_linear_field_has_zero_interior_residual():
    """For u linear on affine elements, (A u)_g = int grad(phi_g).c = 0 at every
    node whose basis function vanishes on the box boundary; GLL quadrature is
    exact for that integrand (degree <= 2N-1)."""
    m = small_mesh((3, 2, 2), 4, L=(1.0, 1.5, 0.7))
    ug = np.zeros(m.n_unique)
    ug[m.l2g] = 0.3 * m.X - 1.2 * m.Y + 2.0 * m.Z + 0.5
    Au = oracle.gather_sum(m, oracle.ax_local(m, oracle.scatter(m, ug)))
    interior = m.mask == 1
    assert np.abs(Au[interior]).max() < 1e-12
    assert np.abs(Au[~interior]).max() > 1e-3


def test_helmholtz_mass_term_only():
    m = small_mesh((2, 1, 1), 3, deform=0.05)
    u = np.random.default_rng(4).standard_normal(m.n_local)
    np.testing.assert_allclose(oracle.ax_local(m, u, 0.0, 2.5), 2.5 * m.B * u, rtol=1e-15)


def test_element_matrices_affine_1d_limit():
    """One unit-cube element at N = 1 (2-point Lobatto rule per direction):
    dphi_0/dr = -1/2 at the two nodes of each edge through vertex 0, so
    A_00 = 3 directions x 2 nodes x (1/2)^2 (2/h)^2 x (h/2)^3 = 3h/4."""
    m = small_mesh((1, 1, 1), 1)
    _, rho, D = gll_numpy(1)
    A, _ = element_matrices(m.X, m.Y, m.Z, rho, D)
    h = 1.0
    assert abs(A[0, 0] - 3 * h / 4) < 1e-15
    d = oracle.diag_assembled(m)
    np.testing.assert_allclose(d, np.diag(A), rtol=1e-14)


def test_element_subset_equals_slices_of_the_whole_mesh():
    """The per-element builder used for spot checks of meshes too large to
    build whole gives, for any list of elements in any order, exactly the
    elements of the whole mesh (same coordinates, G_ab and mass)."""
    import workloads
    w = dataclasses.replace(workloads.AX_GS_64.with_nel((3, 4, 2), name="subset"), N=4)
    m = oracle.mesh_from_workload(w)
    n3 = (w.N + 1) ** 3
    elems = np.array([23, 0, 7, 7, 12, 5], dtype=np.int64)
    X, Y, Z, G, B, D = oracle.element_subset(w, elems)
    idx = (elems[:, None] * n3 + np.arange(n3)[None, :]).ravel()
    assert np.array_equal(X, m.X[idx]) and np.array_equal(Y, m.Y[idx]) and np.array_equal(Z, m.Z[idx])
    assert np.array_equal(G, m.G[:, idx]) and np.array_equal(B, m.B[idx]) and np.array_equal(D, m.D)
