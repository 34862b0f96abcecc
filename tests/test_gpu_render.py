"""GPU parity of the in-situ slice renderer against the oracle (the paper's
boundary-layer and vertical temperature slices with iso-levels, Sec. 5.3 and
Sec. 4.5): slice values within the binary32 bound, RGBA bytes identical except
at pixels whose colour or contour decision lies within rounding of a
threshold, the full-size RBC mesh on sampled pixels, and argument checks;
and the iso-surface overview scene: the resampled grid within the binary32
bound, hit/no-hit, depth and colour agreeing with the oracle's ray march on
all but near-tie pixels."""
import numpy as np
import pytest

import oracle
from oracle import render
import workloads

torch = pytest.importorskip("torch")
import paper_2501_13240_gb300 as sem  # noqa: E402

pytestmark = pytest.mark.gpu


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def field(m):
    u = np.zeros(m.n_unique)
    u[m.l2g] = 0.5 + 0.4 * np.sin(2.1 * m.X + 0.3) * np.cos(1.7 * m.Y) * np.sin(3.0 * m.Z + 0.5)
    return u


def ambiguous(ref, vmin, vmax, iso, tol_v):
    """Pixels whose colour channels or contour decision the binary32 path may
    legitimately take differently (within tol_v of a threshold)."""
    t = np.clip((ref - vmin) / (vmax - vmin), 0.0, 1.0)
    amb = np.abs(t - 0.5) * (vmax - vmin) < tol_v
    for C0, C1, lo in ((render.COOL, render.MID, True), (render.MID, render.WARM, False)):
        f = 2.0 * t - (0.0 if lo else 1.0)
        c = C0 + f[..., None] * (C1 - C0)
        near = np.abs(c - np.floor(c) - 0.5) < 2.0 * 255.0 * tol_v / (vmax - vmin) + 1e-3
        amb |= ((t < 0.5) == lo) & near.any(axis=-1)
    for lvl in iso:
        near = np.abs(ref - lvl) < tol_v
        amb |= near
        amb[:, :-1] |= near[:, 1:]
        amb[:-1, :] |= near[1:, :]
    return amb


MESHES = [
    dict(nel=(4, 3, 5), N=5, periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), z_stretch=2.0),
    dict(nel=(3, 3, 3), N=7, deform_amp=0.05),
    dict(nel=(2, 3, 2), N=4, L=(1.0, 2.0, 0.5), z_stretch=1.3),
]


@pytest.mark.parametrize("spec", MESHES, ids=["rbc_like_N5", "deformed_N7", "boxL_N4"])
@pytest.mark.parametrize("axis,frac", [(2, 0.02), (2, 0.5), (0, 0.37), (1, 1.0)])
def test_slice_matches_oracle(spec, axis, frac):
    om = oracle.box_mesh(**spec)
    gm = sem.sem_mesh_create_box(**spec)
    u = field(om)
    coord = frac * om.L[axis]
    W, H, vmin, vmax, iso = 37, 29, 0.2, 0.8, (0.4, 0.6)
    ref = render.slice_values(om, u, axis, coord, W, H)
    vals, rgba = sem.sem_render_slice(gm, torch.from_numpy(u).cuda(), axis, coord, W, H, vmin, vmax, iso)
    got = host(vals)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 4e-6 * scale
    img = host(rgba)
    want = render.colorize(ref, vmin, vmax, iso)
    diff = np.any(img != want, axis=-1)
    amb = ambiguous(ref, vmin, vmax, iso, 8e-6 * scale)
    assert not np.any(diff & ~amb), np.argwhere(diff & ~amb)[:5]
    assert amb.mean() < 0.05
    gm.destroy()


def test_rbc_32_full_resolution_sampled():
    """The 32^3-element stretched RBC mesh at 4096 x 4096 pixels (the paper's
    image size), checked at 300 sampled pixels of a boundary-layer slice."""
    w = workloads.RBC_32
    om = oracle.box_mesh(w.nel, w.N, w.L, w.periodic, w.dirichlet, w.z_stretch, geometry=False)
    gm = sem.mesh_from_workload(w)
    u = field(om)
    W = H = 4096
    vals, rgba = sem.sem_render_slice(gm, torch.from_numpy(u).cuda(), 2, 0.01, W, H, 0.2, 0.8, (0.5,))
    got = host(vals)
    rng = np.random.default_rng(9)
    pix = [(int(x), int(y)) for x, y in zip(rng.integers(0, W, 300), rng.integers(0, H, 300))]
    ref = render.slice_values(om, u, 2, 0.01, W, H, pixels=pix)
    sub = np.array([got[y, x] for x, y in pix])
    assert np.abs(sub - ref).max() <= 4e-6 * np.abs(ref).max()
    img = host(rgba)
    assert img[..., 3].min() == 255
    gm.destroy()


def test_edges_and_invalid_arguments(tmp_path):
    spec = MESHES[0]
    om = oracle.box_mesh(**spec)
    gm = sem.sem_mesh_create_box(**spec)
    u = field(om)
    ud = torch.from_numpy(u).cuda()
    for axis, coord in ((2, 0.0), (2, 1.0), (0, 1.0)):  # boundary planes
        vals, _ = sem.sem_render_slice(gm, ud, axis, coord, 5, 3)
        ref = render.slice_values(om, u, axis, coord, 5, 3)
        assert np.abs(host(vals) - ref).max() <= 4e-6 * np.abs(ref).max()
    vals, rgba = sem.sem_render_slice(gm, ud, 1, 0.5, 1, 1)  # one pixel
    assert np.isfinite(host(vals)).all()
    for bad in (dict(axis=3, coord=0.5), dict(axis=2, coord=1.5), dict(axis=2, coord=-0.1)):
        with pytest.raises(sem.SemError):
            sem.sem_render_slice(gm, ud, bad["axis"], bad["coord"], 4, 4)
    with pytest.raises(sem.SemError):
        sem.sem_render_slice(gm, ud, 2, 0.5, 4, 4, vmin=1.0, vmax=1.0)
    with pytest.raises(sem.SemError):
        sem.sem_render_slice(gm, ud, 2, 0.5, 0, 4)
    _, rgba = sem.sem_render_slice(gm, ud, 2, 0.5, 8, 6, 0.2, 0.8, (0.5,))
    path = tmp_path / "slice.ppm"
    sem.sem_write_ppm(str(path), host(rgba))
    data = path.read_bytes()
    assert data.startswith(b"P6\n8 6\n255\n") and len(data) == len(b"P6\n8 6\n255\n") + 8 * 6 * 3
    gm.destroy()


# ------------------------------------------------------------ 3-D scene

def scene_field(m):
    u = np.zeros(m.n_unique)
    u[m.l2g] = 1.0 - m.Z / m.L[2] + 0.15 * np.sin(3.1 * m.X + 0.4) * np.cos(2.3 * m.Y) * np.sin(np.pi * m.Z / m.L[2])
    return u


@pytest.mark.parametrize("spec", MESHES[:2], ids=["rbc_like_N5", "deformed_N7"])
def test_scene_matches_oracle(spec):
    om = oracle.box_mesh(**spec)
    gm = sem.sem_mesh_create_box(**spec)
    u = scene_field(om)
    R, W, H = (14, 12, 16), 40, 30
    cam = dict(eye=(2.2, -1.6, 1.4), target=(0.5, 0.5, 0.45), up=(0.0, 0.0, 1.0), fov_deg=35.0)
    vol, depth, rgba = sem.sem_render_scene(gm, torch.from_numpy(u).cuda(), cam["eye"], cam["target"], cam["up"],
                                            cam["fov_deg"], W, H, R, 0.0, 1.0, (0.4, 0.6))
    ref_vol = render.resample(om, u, R)
    assert np.abs(host(vol) - ref_vol).max() <= 4e-6 * np.abs(ref_vol).max()
    ref_d, ref_img = render.render_scene(ref_vol, om.L, cam["eye"], cam["target"], cam["up"], cam["fov_deg"], W, H,
                                         0.0, 1.0, (0.4, 0.6))
    d, img = host(depth), host(rgba)
    h = min(om.L[q] / R[q] for q in range(3))
    same_status = (d >= 0) == (ref_d >= 0)
    assert same_status.mean() >= 0.98
    both = same_status & (d >= 0)
    assert both.sum() > 0.08 * W * H  # the levels are in view (top of the box)
    close = np.abs(d - ref_d) <= 1e-3 * h
    assert close[both].mean() >= 0.98
    chan = np.abs(img.astype(int) - ref_img.astype(int)).max(axis=-1)
    assert (chan[same_status & (close | (d < 0))] <= 1).mean() >= 0.98
    assert (img[..., 3] == 255).all()
    gm.destroy()


def test_scene_background_and_arguments():
    spec = MESHES[0]
    gm = sem.sem_mesh_create_box(**spec)
    u = torch.ones(gm.n_unique, dtype=torch.float64, device="cuda") * 0.25
    _, depth, rgba = sem.sem_render_scene(gm, u, (3.0, 3.0, 3.0), (6.0, 6.0, 6.0), (0, 0, 1), 40.0, 8, 6, (4, 4, 4))
    assert (host(depth) == -1).all() and (host(rgba) == 255).all()
    with pytest.raises(sem.SemError):
        sem.sem_render_scene(gm, u, (0.5, 0.5, 3.0), (0.5, 0.5, 3.0), (0, 0, 1), 40.0, 8, 6, (4, 4, 4))  # eye = target
    with pytest.raises(sem.SemError):
        sem.sem_render_scene(gm, u, (0.5, 0.5, 3.0), (0.5, 0.5, 0.0), (0, 0, 1), 40.0, 8, 6, (4, 4, 4))  # up || view
    with pytest.raises(sem.SemError):
        sem.sem_render_scene(gm, u, (0.5, 0.5, 3.0), (0.5, 0.5, 0.0), (0, 1, 0), 40.0, 8, 6, (0, 4, 4))
    gm.destroy()
