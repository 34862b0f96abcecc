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


# ------------------------------------------------------------ 3-D scene pins

def test_resample_reproduces_polynomials():
    m = oracle.box_mesh((2, 3, 2), 4, L=(1.0, 2.0, 0.5), z_stretch=1.5)
    u = nodal(m, poly)
    R = (7, 9, 5)
    vol = render.resample(m, u, R)
    x = (np.arange(R[0]) + 0.5) * m.L[0] / R[0]
    y = (np.arange(R[1]) + 0.5) * m.L[1] / R[1]
    z = (np.arange(R[2]) + 0.5) * m.L[2] / R[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    np.testing.assert_allclose(vol, poly(X, Y, Z), rtol=0, atol=1e-12)


def test_trilinear_is_exact_for_linear_fields():
    L = (1.0, 2.0, 0.5)
    R = (5, 6, 4)
    lin = lambda x, y, z: 0.3 * x - 1.2 * y + 2.0 * z + 0.7  # noqa: E731
    cz, cy, cx = np.meshgrid(*[(np.arange(R[d]) + 0.5) * L[d] / R[d] for d in (2, 1, 0)], indexing="ij")
    vol = lin(cx, cy, cz)
    rng = np.random.default_rng(3)
    for _ in range(50):  # interior points: at least half a cell from the walls
        p = [rng.uniform(0.5 * L[d] / R[d], L[d] - 0.5 * L[d] / R[d]) for d in range(3)]
        assert render.trilinear(vol, L, p) == pytest.approx(lin(*p), abs=1e-13)


def test_scene_hits_a_level_plane_straight_below_the_eye():
    # u = z and the level 0.5: straight down from the eye the hit is at z = 0.5
    m = oracle.box_mesh((2, 2, 2), 3)
    vol = render.resample(m, nodal(m, lambda x, y, z: z + 0.0 * x), (8, 8, 8))
    eye = (0.5, 0.5, 2.0)
    depth, img = render.render_scene(vol, m.L, eye, (0.5, 0.5, 0.0), (0.0, 1.0, 0.0), 30.0, 9, 7, 0.0, 1.0, [0.5])
    assert depth[3, 4] == pytest.approx(1.5, abs=1e-12)  # the central pixel's ray is -z
    assert np.allclose(depth, depth[::-1, ::-1])         # symmetric view, symmetric depth
    assert (depth > 0).all()                             # every ray meets the plane inside the box
    c = render.colour(0.5, 0.0, 1.0)                     # the level's colour, dimmed by the depth cue
    s = img[3, 4, :3] / c
    assert 0.5 - 1e-2 <= s.min() and s.max() <= 1.0 + 1e-2 and np.ptp(s) < 0.02


def test_scene_background_and_walls():
    m = oracle.box_mesh((2, 2, 2), 3)
    vol = render.resample(m, nodal(m, lambda x, y, z: 0.25 + 0.0 * x), (6, 6, 6))
    depth, img = render.render_scene(vol, m.L, (3.0, 3.0, 3.0), (6.0, 6.0, 6.0), (0, 0, 1), 40.0, 8, 6, 0.0, 1.0,
                                     [0.5])
    assert (depth == -1).all() and (img == 255).all()     # looking away from the box
    depth, img = render.render_scene(vol, m.L, (0.5, 0.5, 3.0), (0.5, 0.5, 0.0), (0, 1, 0), 10.0, 5, 5, 0.0, 1.0,
                                     [0.5])
    wall = np.floor(render.colour(0.25, 0.0, 1.0) * 0.35 + 0.5)
    assert (depth == -1).all() and (img[..., :3] == wall).all()  # no crossing: the dimmed walls
