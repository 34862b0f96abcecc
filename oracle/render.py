"""Oracle of the in-situ slice rendering (TEST INFRASTRUCTURE ONLY).

The paper's in-situ scenes (Sec. 5.3 and the figures of Sec. 4.5) are
temperature slices through the boundary layers near the plates, vertical
slices, and iso-levels T = 0.4 and 0.6, rendered from data resident on the
GPU. Readings (the paper fixes only the scene content):

* a slice is the plane x_a = c (a = 0, 1, 2) of the undeformed box; the image
  spans the two other axes in increasing order (a = 0: y, z; a = 1: x, z;
  a = 2: x, y), width W along the first, height H along the second, pixel
  (px, py) centred at ((px + 1/2) L_first / W, (py + 1/2) L_second / H), row
  py = 0 at the low end, stored row-major [py][px];
* a coordinate x along an axis with element interfaces x_0 < ... < x_n
  (uniform, or the tanh interfaces of the stretched z axis) lies in element
  k = the largest with x_k <= x (at most n - 1), local coordinate
  xi = 2 (x - x_k) / (x_{k+1} - x_k) - 1; on a deformed mesh this is the
  reference location, not the physical one;
* the value is the SEM polynomial of the element there:
  v = sum_{ijk} u(e; i, j, k) l_i(xi) l_j(eta) l_k(zeta), l_m the Lagrange
  basis on the GLL nodes;
* colour: t = clamp((v - vmin) / (vmax - vmin), 0, 1), piecewise linear in
  RGB through blue (59, 76, 192) at t = 0, grey (221, 221, 221) at t = 1/2
  and red (180, 4, 38) at t = 1 (the end and middle colours of Moreland's
  cool-warm map), channel = floor(c + 1/2), alpha 255; NaN is magenta;
* contour lines: a pixel is black when, for some level l, v - l >= 0 at the
  pixel and < 0 at its right or upper neighbour, or the other way round.
Everything here is binary64.
"""
from __future__ import annotations

import numpy as np

from . import Mesh

COOL = np.array([59.0, 76.0, 192.0])
MID = np.array([221.0, 221.0, 221.0])
WARM = np.array([180.0, 4.0, 38.0])


def interfaces(m: Mesh, axis: int) -> np.ndarray:
    """Element interfaces along one axis of the undeformed box."""
    n = m.nel[axis]
    L = m.L[axis]
    k = np.arange(n + 1, dtype=np.float64)
    if axis == 2 and m.z_stretch > 0.0:
        s = m.z_stretch
        return 0.5 * L * (1.0 + np.tanh(s * (2.0 * k / n - 1.0)) / np.tanh(s))
    return k * L / n


def locate(xk: np.ndarray, x: np.ndarray):
    """(element index, local coordinate in [-1, 1]) of coordinates x."""
    n = len(xk) - 1
    k = np.clip(np.searchsorted(xk, x, side="right") - 1, 0, n - 1)
    xi = 2.0 * (x - xk[k]) / (xk[k + 1] - xk[k]) - 1.0
    return k, xi


def lagrange(nodes: np.ndarray, s: np.ndarray) -> np.ndarray:
    """[len(s), len(nodes)]: l_m(s) on the given nodes."""
    out = np.ones((len(s), len(nodes)))
    for mth in range(len(nodes)):
        for q in range(len(nodes)):
            if q != mth:
                out[:, mth] *= (s - nodes[q]) / (nodes[mth] - nodes[q])
    return out


def in_plane_axes(axis: int):
    return [a for a in range(3) if a != axis]


def slice_values(m: Mesh, u_g: np.ndarray, axis: int, coord: float, W: int, H: int, pixels=None) -> np.ndarray:
    """[H, W] values of the unique-node field u_g on the slice, or the values
    at the listed (px, py) pixels only (for images too large to evaluate
    whole here)."""
    n = m.N + 1
    a, b = in_plane_axes(axis)
    whole = pixels is None
    if whole:
        pixels = [(px, py) for py in range(H) for px in range(W)]
    px = np.array([p[0] for p in pixels], dtype=np.int64)
    py = np.array([p[1] for p in pixels], dtype=np.int64)
    ka, sa = locate(interfaces(m, a), (px + 0.5) * m.L[a] / W)
    kb, sb = locate(interfaces(m, b), (py + 0.5) * m.L[b] / H)
    kc, sc = locate(interfaces(m, axis), np.array([coord], dtype=np.float64))
    la, lb, lc = lagrange(m.xi, sa), lagrange(m.xi, sb), lagrange(m.xi, sc)[0]
    out = np.zeros(len(pixels))
    for t in range(len(pixels)):
        ek = [0, 0, 0]
        ek[a], ek[b], ek[axis] = ka[t], kb[t], kc[0]
        e = ek[0] + m.nel[0] * (ek[1] + m.nel[1] * ek[2])
        ue = u_g[m.l2g[e * n ** 3:(e + 1) * n ** 3]].reshape(n, n, n)  # [k, j, i]
        basis = [None, None, None]
        basis[a], basis[b], basis[axis] = la[t], lb[t], lc
        # v = sum_{ijk} u[k, j, i] l_i(x) l_j(y) l_k(z)
        out[t] = np.einsum("kji,i,j,k->", ue, basis[0], basis[1], basis[2])
    return out.reshape(H, W) if whole else out


def colorize(v: np.ndarray, vmin: float, vmax: float, iso=()) -> np.ndarray:
    """[H, W, 4] uint8 image of the values (colour map and contour lines)."""
    t = np.clip((v - vmin) / (vmax - vmin), 0.0, 1.0)
    lo = t < 0.5
    f = np.where(lo, 2.0 * t, 2.0 * t - 1.0)[..., None]
    c = np.where(lo[..., None], COOL + f * (MID - COOL), MID + f * (WARM - MID))
    rgb = np.floor(np.nan_to_num(c) + 0.5).astype(np.uint8)
    rgb[np.isnan(v)] = (255, 0, 255)
    img = np.concatenate([rgb, np.full(v.shape + (1,), 255, np.uint8)], axis=-1)
    H, W = v.shape
    line = np.zeros((H, W), dtype=bool)
    for lvl in iso:
        s = v - lvl >= 0.0
        d = s[:, :-1] != s[:, 1:]
        line[:, :-1] |= d
        d = s[:-1, :] != s[1:, :]
        line[:-1, :] |= d
    img[line] = (0, 0, 0, 255)
    return img
