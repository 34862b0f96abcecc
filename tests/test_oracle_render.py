"""Pins of the oracle's slice rendering: exact reproduction of polynomials of
degree <= N per direction at the pixel centres (locates, Lagrange basis,
element numbering and axis order), the colour map at its control points, the
contour rule on a linear field, and the image orientation. CPU only."""
import numpy as np
import pytest

import oracle
from oracle import render


def poly(x, y, z):
    return x ** 3 - 2.0 * x * y ** 2 + z ** 4 + 0.5 * y * z - 1.0


def nodal(m, f):
    u = np.zeros(m.n_unique)
    u[m.l2g] = f(m.X, m.Y, m.Z)
    return u


@pytest.mark.parametrize("axis,coord", [(0, 0.37), (1, 1.21), (2, 0.083), (2, 0.5)])
def test_slice_reproduces_polynomials(axis, coord):
    m = oracle.box_mesh((2, 3, 2), 4, L=(1.0, 2.0, 0.5), z_stretch=1.5)
    u = nodal(m, poly)
    W, H = 13, 11
    v = render.slice_values(m, u, axis, coord, W, H)
    a, b = render.in_plane_axes(axis)
    xa = (np.arange(W) + 0.5) * m.L[a] / W
    xb = (np.arange(H) + 0.5) * m.L[b] / H
    P = [None, None, None]
    P[a] = xa[None, :]
    P[b] = xb[:, None]
    P[axis] = coord
    np.testing.assert_allclose(v, poly(P[0], P[1], P[2]) + 0.0 * v, rtol=0, atol=1e-12)


def test_slice_at_nodes_returns_nodal_values():
    # a plane through GLL nodes of a uniform mesh: values at pixel centres that
    # fall on nodes equal the nodal values (N = 2: nodes at element ends and midpoints)
    m = oracle.box_mesh((2, 2, 2), 2)
    u = np.random.default_rng(5).standard_normal(m.n_unique)
    v = render.slice_values(m, u, 2, 0.25, 4, 4)  # pixel centres 0.125, 0.375, ...: not nodes
    assert np.all(np.isfinite(v))
    # z = 0.25 is the midpoint node of the first element layer; x = y = 0.25 too with W = H = 2
    v2 = render.slice_values(m, u, 2, 0.25, 2, 2)
    n = 3
    e, ijk = 0, 1 + n * 1 + n * n * 1  # element 0, local node (1, 1, 1)
    assert v2[0, 0] == pytest.approx(u[m.l2g[e * n ** 3 + ijk]], abs=1e-14)


def test_colour_map_control_points():
    v = np.array([[0.0, 0.5, 1.0, 0.25, -3.0, 7.0, np.nan]])
    img = render.colorize(v, 0.0, 1.0)
    assert img[0, 0].tolist() == [59, 76, 192, 255]
    assert img[0, 1].tolist() == [221, 221, 221, 255]
    assert img[0, 2].tolist() == [180, 4, 38, 255]
    assert img[0, 3].tolist() == [140, 149, 207, 255]  # halfway blue -> grey: (140, 148.5, 206.5) rounded
    assert img[0, 4].tolist() == [59, 76, 192, 255]    # clamped
    assert img[0, 5].tolist() == [180, 4, 38, 255]
    assert img[0, 6].tolist() == [255, 0, 255, 255]


def test_contour_of_a_linear_field_and_orientation():
    m = oracle.box_mesh((2, 2, 2), 3)
    u = nodal(m, lambda x, y, z: x + 0.0 * y)
    v = render.slice_values(m, u, 2, 0.5, 10, 6)
    img = render.colorize(v, 0.0, 1.0, iso=[0.5])
    black = np.all(img[..., :3] == 0, axis=-1)
    assert black[:, 4].all() and black.sum() == 6  # between x = 0.45 and 0.55, the lower pixel
    # vertical slice x = 0.3 of u = z: rows increase with z (row 0 at the bottom)
    u = nodal(m, lambda x, y, z: z + 0.0 * x)
    v = render.slice_values(m, u, 0, 0.3, 5, 8)
    assert np.all(np.diff(v[:, 2]) > 0) and np.allclose(v[:, 0], v[:, 4])
