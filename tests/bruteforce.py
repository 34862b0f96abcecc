"""Dense brute-force spectral-element matrices for tiny meshes (tests only).

Built independently of the oracle's sum-factorised loops: the 1-D derivative
matrix comes from numpy's Legendre Vandermonde matrices, element matrices are
formed as dense Kronecker products with the inverse Jacobian from
numpy.linalg.inv at every quadrature point, and the assembly uses an explicit
0/1 matrix Q built from node coordinates.
"""
import numpy as np
import numpy.polynomial.legendre as npl


def gll_numpy(N):
    """GLL nodes from numpy's roots of P_N', weights from the moment
    equations, D = V' V^-1."""
    inner = np.sort(npl.Legendre.basis(N).deriv().roots().real)
    xi = np.concatenate([[-1.0], inner, [1.0]])
    V = npl.legvander(xi, N)
    rhs = np.zeros(N + 1)
    rhs[0] = 2.0
    rho = np.linalg.solve(V.T, rhs)
    dV = np.stack([npl.legval(xi, npl.legder(np.eye(N + 1)[k])) for k in range(N + 1)], axis=1)
    D = np.linalg.solve(V.T, dV.T).T
    return xi, rho, D


def element_matrices(Xe, Ye, Ze, rho, D):
    """Dense stiffness A_e = sum_c (d phi/dx_c)^T W |J| (d phi/dx_c) and the
    diagonal mass B_e at GLL quadrature, local order p = i + n j + n^2 k."""
    n = D.shape[0]
    I = np.eye(n)
    Dr = np.kron(I, np.kron(I, D))
    Ds = np.kron(I, np.kron(D, I))
    Dt = np.kron(D, np.kron(I, I))
    grads = (Dr, Ds, Dt)
    Jm = np.zeros((n ** 3, 3, 3))
    for c, xc in enumerate((Xe, Ye, Ze)):
        for a in range(3):
            Jm[:, c, a] = grads[a] @ xc
    det = np.linalg.det(Jm)
    R = np.linalg.inv(Jm)  # R[q, a, c] = d r_a / d x_c
    w = np.kron(np.kron(rho, rho), rho) * det
    A = np.zeros((n ** 3, n ** 3))
    for c in range(3):
        Gc = sum(R[:, a, c][:, None] * grads[a] for a in range(3))
        A += Gc.T @ (w[:, None] * Gc)
    return A, w


def unique_classes(coords, L, periodic, scale=1e9):
    """Equivalence classes of local nodes by coordinate (periodic wrap)."""
    key = []
    for d in range(3):
        c = np.asarray(coords[d], dtype=np.float64).copy()
        if periodic[d]:
            c = np.mod(c, L[d])
            c[np.isclose(c, L[d], atol=1e-12)] = 0.0
        key.append(np.round(c * scale).astype(np.int64))
    key = np.stack(key, axis=1)
    _, cls = np.unique(key, axis=0, return_inverse=True)
    return cls.ravel()


def assembly_matrix(l2g, n_unique):
    Q = np.zeros((len(l2g), n_unique))
    Q[np.arange(len(l2g)), l2g] = 1.0
    return Q


def dense_global(mesh, h1=1.0, h2=0.0):
    """Q^T (h1 A_L + h2 B_L) Q with per-element dense blocks (unmasked)."""
    n3 = (mesh.N + 1) ** 3
    _, rho, D = gll_numpy(mesh.N)
    AL = np.zeros((mesh.n_local, mesh.n_local))
    for e in range(mesh.E):
        s = slice(e * n3, (e + 1) * n3)
        A, w = element_matrices(mesh.X[s], mesh.Y[s], mesh.Z[s], rho, D)
        AL[s, s] = h1 * A + h2 * np.diag(w)
    Q = assembly_matrix(mesh.l2g, mesh.n_unique)
    return Q.T @ AL @ Q, AL, Q
