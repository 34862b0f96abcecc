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


# ---------------------------------------------------------------- 3-D scene
# Readings for the overview scene (iso-surfaces T = 0.4, 0.6 in perspective,
# with the box walls behind them):
# * the field is resampled at the cell centres of an R_x x R_y x R_z grid of
#   the undeformed box (x_i = (i + 1/2) L_x / R_x), each value the SEM
#   polynomial there, and read back by trilinear interpolation (index
#   coordinate g = x R / L - 1/2, clamped to [0, R - 1]);
# * pinhole camera: f = (target - eye)/|.|, r = (f x up)/|.|, u = r x f; the
#   ray through pixel (px, py) has direction f + s_x r + s_y u normalised,
#   s_x = (2 (px + 1/2)/W - 1) tan(fov/2) W/H, s_y = (2 (py + 1/2)/H - 1)
#   tan(fov/2) (row 0 at the bottom);
# * the ray enters and leaves the box at t0 = max(0, slab entries) and t1 =
#   min(slab exits); no intersection: white, depth -1;
# * samples at t0 + s h, h = min_d L_d / R_d, s = 0 .. floor((t1 - t0)/h);
#   the first sample interval in which v - level changes sign (>= 0 against
#   < 0) for some level is the hit, at t = t_{s-1} + h a/(a - b) (a, b the
#   values of v - level at the two ends), the earliest such t among levels;
#   its colour is the colour map at the level, times the depth cue
#   1 - (t - t_near)/(2 (t_far - t_near)) clamped to [1/2, 1] (t_near, t_far:
#   nearest and farthest box corner from the eye); depth = t;
# * a ray through the box without a hit shows the colour map of the last
#   sample times 0.35 (the walls behind); depth -1.

def resample(m: Mesh, u_g: np.ndarray, R) -> np.ndarray:
    """[R_z, R_y, R_x] values of the field at the cell centres."""
    n = m.N + 1
    ks, ls = [], []
    for d in range(3):
        x = (np.arange(R[d]) + 0.5) * m.L[d] / R[d]
        k, s = locate(interfaces(m, d), x)
        ks.append(k)
        ls.append(lagrange(m.xi, s))
    uL = u_g[m.l2g].reshape(m.E, n, n, n)  # [e, k, j, i]
    out = np.zeros((R[2], R[1], R[0]))
    for c in range(R[2]):
        for b in range(R[1]):
            for a in range(R[0]):
                e = ks[0][a] + m.nel[0] * (ks[1][b] + m.nel[1] * ks[2][c])
                out[c, b, a] = np.einsum("kji,i,j,k->", uL[e], ls[0][a], ls[1][b], ls[2][c])
    return out


def trilinear(vol: np.ndarray, L, p) -> float:
    R = (vol.shape[2], vol.shape[1], vol.shape[0])
    i0, f = [0, 0, 0], [0.0, 0.0, 0.0]
    for d in range(3):
        g = min(max(p[d] * R[d] / L[d] - 0.5, 0.0), R[d] - 1.0)
        i0[d] = min(int(np.floor(g)), R[d] - 2) if R[d] > 1 else 0
        f[d] = g - i0[d] if R[d] > 1 else 0.0
    v = 0.0
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = (f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) * (f[2] if dz else 1 - f[2])
                if w != 0.0:
                    v += w * vol[i0[2] + dz, i0[1] + dy, i0[0] + dx]
    return v


def colour(v: float, vmin: float, vmax: float) -> np.ndarray:
    t = min(max((v - vmin) / (vmax - vmin), 0.0), 1.0)
    if t < 0.5:
        return COOL + 2.0 * t * (MID - COOL)
    return MID + (2.0 * t - 1.0) * (WARM - MID)


def render_scene(vol: np.ndarray, L, eye, target, up, fov_deg, W, H, vmin, vmax, iso, pixels=None):
    """(depth [H, W], rgba [H, W, 4]) of the iso-surface scene, or the values
    at the listed pixels only."""
    eye, target, up = (np.asarray(v, dtype=np.float64) for v in (eye, target, up))
    fw = target - eye
    fw /= np.linalg.norm(fw)
    rt = np.cross(fw, up)
    rt /= np.linalg.norm(rt)
    uu = np.cross(rt, fw)
    tanh_ = np.tan(np.radians(fov_deg) / 2.0)
    R = (vol.shape[2], vol.shape[1], vol.shape[0])
    h = min(L[d] / R[d] for d in range(3))
    corners = [np.array([x, y, z]) for x in (0.0, L[0]) for y in (0.0, L[1]) for z in (0.0, L[2])]
    dist = [float(np.linalg.norm(c - eye)) for c in corners]
    tn, tf = min(dist), max(dist)
    whole = pixels is None
    if whole:
        pixels = [(px, py) for py in range(H) for px in range(W)]
    depth = np.full(len(pixels), -1.0)
    rgba = np.zeros((len(pixels), 4), dtype=np.uint8)
    for q, (px, py) in enumerate(pixels):
        sx = (2.0 * (px + 0.5) / W - 1.0) * tanh_ * W / H
        sy = (2.0 * (py + 0.5) / H - 1.0) * tanh_
        dr = fw + sx * rt + sy * uu
        dr /= np.linalg.norm(dr)
        t0, t1 = 0.0, np.inf
        for d in range(3):
            if dr[d] != 0.0:
                ta, tb = (0.0 - eye[d]) / dr[d], (L[d] - eye[d]) / dr[d]
                t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
            elif not (0.0 <= eye[d] <= L[d]):
                t1 = -1.0
        if t1 < t0:
            rgba[q] = (255, 255, 255, 255)
            continue
        S = int(np.floor((t1 - t0) / h))
        prev = trilinear(vol, L, eye + t0 * dr)
        hit = None
        for s in range(1, S + 1):
            ts = t0 + s * h
            cur = trilinear(vol, L, eye + ts * dr)
            best = None
            for lvl in iso:
                a, b = prev - lvl, cur - lvl
                if (a >= 0.0) != (b >= 0.0):
                    tq = ts - h + h * a / (a - b)
                    if best is None or tq < best[0]:
                        best = (tq, lvl)
            if best is not None:
                hit = best
                break
            prev = cur
        if hit is not None:
            shade = min(max(1.0 - (hit[0] - tn) / (2.0 * (tf - tn)), 0.5), 1.0)
            c = colour(hit[1], vmin, vmax) * shade
            depth[q] = hit[0]
        else:
            c = colour(prev, vmin, vmax) * 0.35
        rgba[q, :3] = np.floor(c + 0.5).astype(np.uint8)
        rgba[q, 3] = 255
    if whole:
        return depth.reshape(H, W), rgba.reshape(H, W, 4)
    return depth, rgba
