"""Pins of the oracle's GLL basis (Sec. 2.2: nodal GLL basis, (p+1)x(p+1)
operator matrices) against closed forms, quadrature exactness and numpy's
Legendre routines. CPU only."""
import numpy as np
import numpy.polynomial.legendre as npl
import pytest

import oracle


@pytest.mark.parametrize("N", range(1, 13))
def test_nodes_match_numpy_legendre_roots(N):
    xi, rho, D = oracle.gll(N)
    inner = np.sort(npl.Legendre.basis(N).deriv().roots().real)
    assert xi[0] == -1.0 and xi[-1] == 1.0
    np.testing.assert_allclose(xi[1:-1], inner, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(xi, -xi[::-1])  # exact symmetry


@pytest.mark.parametrize("N", range(1, 13))
def test_weights_solve_moment_equations(N):
    """rho solves sum_i rho_i P_k(xi_i) = int P_k = 2 delta_k0, k = 0..N
    (numpy Legendre Vandermonde + linalg.solve)."""
    xi, rho, _ = oracle.gll(N)
    V = npl.legvander(xi, N).T  # V[k, i] = P_k(xi_i)
    rhs = np.zeros(N + 1)
    rhs[0] = 2.0
    np.testing.assert_allclose(rho, np.linalg.solve(V, rhs), rtol=1e-13, atol=1e-15)
    assert abs(rho.sum() - 2.0) < 1e-14


@pytest.mark.parametrize("N", range(1, 13))
def test_quadrature_exact_to_degree_2N_minus_1(N):
    xi, rho, _ = oracle.gll(N)
    for k in range(0, 2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(rho, xi ** k) - exact) < 1e-13, k
    # and not exact at degree 2N (the GLL rule has degree 2N-1)
    assert abs(np.dot(rho, xi ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-9


@pytest.mark.parametrize("N", range(1, 13))
def test_derivative_matrix_exact_on_polynomials(N):
    xi, _, D = oracle.gll(N)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-12 * N * N)
    for m in range(1, N + 1):
        np.testing.assert_allclose(D @ xi ** m, m * xi ** (m - 1), rtol=0, atol=5e-13 * N * N)


@pytest.mark.parametrize("N", range(1, 13))
def test_derivative_matrix_matches_vandermonde(N):
    """D = V' V^{-1} with the Legendre Vandermonde matrices (numpy)."""
    xi, _, D = oracle.gll(N)
    V = npl.legvander(xi, N)
    dV = np.stack([npl.legval(xi, npl.legder(np.eye(N + 1)[k])) for k in range(N + 1)], axis=1)
    np.testing.assert_allclose(D, np.linalg.solve(V.T, dV.T).T, rtol=0, atol=1e-11 * N * N)


def test_closed_forms_N1_N2():
    xi, rho, D = oracle.gll(1)
    np.testing.assert_array_equal(xi, [-1.0, 1.0])
    np.testing.assert_allclose(rho, [1.0, 1.0], rtol=1e-15)
    np.testing.assert_allclose(D, [[-0.5, 0.5], [-0.5, 0.5]], rtol=1e-15)
    xi, rho, D = oracle.gll(2)
    np.testing.assert_array_equal(xi, [-1.0, 0.0, 1.0])
    np.testing.assert_allclose(rho, [1 / 3, 4 / 3, 1 / 3], rtol=1e-15)
    np.testing.assert_allclose(D, [[-1.5, 2.0, -0.5], [-0.5, 0.0, 0.5], [0.5, -2.0, 1.5]], rtol=1e-15, atol=1e-15)


def test_centro_antisymmetry():
    """D[N-i, N-j] = -D[i, j] (symmetric nodes), the property the even-odd
    split of the contractions relies on."""
    for N in range(1, 13):
        _, _, D = oracle.gll(N)
        np.testing.assert_allclose(D[::-1, ::-1], -D, atol=1e-13 * N * N)


def test_bad_order_rejected():
    with pytest.raises(ValueError):
        oracle.gll(0)
