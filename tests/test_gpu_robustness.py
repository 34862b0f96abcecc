"""Failure detection without a memory checker or a GPU fault: host-side audits
of every index table, faults injected into the tables on the host side of the
API and caught by the audit, canary padding around every output buffer (no
entry point writes outside the bytes it owns), a non-SPD Helmholtz request,
and truncated checkpoint files."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
import paper_2501_13240_gb300 as sem  # noqa: E402
from paper_2501_13240_gb300 import adjoint as gadj  # noqa: E402

pytestmark = pytest.mark.gpu

MESHES = [dict(nel=(5, 3, 3), N=7, deform_amp=0.05), dict(nel=(2, 3, 4), N=9, periodic=(1, 1, 0),
                                                           dirichlet=(0, 0, 0, 0, 1, 1), z_stretch=2.0),
          dict(nel=(3, 3, 2), N=2, periodic=(1, 0, 1), dirichlet=(0, 0, 1, 1, 0, 0)), dict(nel=(4, 3, 2), N=1),
          dict(nel=(2, 2, 2), N=10, periodic=(1, 1, 1), dirichlet=(0,) * 6)]

PAD = 64
BYTE = 0x5A


def padded(n, dtype, fill=None):
    """(whole buffer, the middle view handed to the library)"""
    item = torch.empty(0, dtype=dtype).element_size()
    raw = torch.full(((n + 2 * PAD) * item,), BYTE, dtype=torch.uint8, device="cuda")
    whole = raw.view(dtype)
    mid = whole[PAD:PAD + n]
    if fill is not None:
        mid.copy_(fill)
    return raw, mid


def canaries_intact(raw, n, dtype):
    item = torch.empty(0, dtype=dtype).element_size()
    torch.cuda.synchronize()
    b = raw.cpu().numpy()
    return bool((b[:PAD * item] == BYTE).all() and (b[(PAD + n) * item:] == BYTE).all())


@pytest.mark.parametrize("spec", MESHES, ids=["deformed_N7", "rbc_N9", "periodic_N2", "N1", "allperiodic_N10"])
def test_mesh_tables_pass_the_audit(spec):
    gm = sem.sem_mesh_create_box(**spec)
    sem.sem_mesh_validate(gm)
    gm.destroy()


def test_audit_catches_injected_table_faults():
    for where in ("l2g", "mask"):
        gm = sem.sem_mesh_create_box((3, 2, 2), 3)
        info = gm.info
        if where == "l2g":
            t = torch.as_tensor(sem._DeviceView(info.l2g, gm.n_local, "<i4"), device="cuda")
            t[17] = gm.n_unique + 5  # out of range
            msg = "out of range"
        else:
            t = torch.as_tensor(sem._DeviceView(info.mask, gm.n_unique, "|u1"), device="cuda")
            t[0] = 1 - int(t[0])  # mask no longer matches l2gm
            msg = "l2gm"
        torch.cuda.synchronize()
        with pytest.raises(sem.SemError) as ei:
            sem.sem_mesh_validate(gm)
        assert msg in str(ei.value)
        gm.destroy()  # the corrupted mesh is never used by a kernel


def test_no_entry_point_writes_outside_its_buffers():
    spec = dict(nel=(3, 3, 3), N=5, periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), z_stretch=1.5)
    gm = sem.sem_mesh_create_box(**spec)
    nL, nU = gm.n_local, gm.n_unique
    f64 = torch.float64
    u = torch.from_numpy(workloads.unique_field(nU, seed=1) * gm.maps()[1]).cuda()
    uL = torch.empty(nL, dtype=f64, device="cuda")
    sem.sem_scatter(gm, u, uL)
    checks = []

    def out(n, dtype=f64, fill=None):
        raw, mid = padded(n, dtype, fill)
        checks.append((raw, n, dtype))
        return mid

    for prec in (sem.SEM_PREC_FP64, sem.SEM_PREC_DF64):
        sem.sem_ax_apply(gm, 1.0, 0.5, uL, out(nL), precision=prec)
        sem.sem_ax_assembled(gm, 1.0, 0.5, u, out(nU), precision=prec)
        sem.sem_ax_assembled_add(gm, 1.0, 0.5, u, out(nU, fill=torch.zeros(nU, dtype=f64)), precision=prec)
        sem.sem_pcg_solve(gm, 1.0, 0.5, u, out(nU), tol=1e-8, precision=prec)
    sem.sem_gs_op(gm, out(nL, fill=uL), True)
    sem.sem_gather(gm, uL, out(nU))
    sem.sem_scatter(gm, u, out(nL))
    sem.sem_jacobi_inv(gm, 1.0, 0.5, out(nU))
    sem.sem_weak_rhs(gm, uL, out(nU))
    P = sem.sem_pmg_create(gm, orders=(5, 2, 1), coarse_tol=1e-2, mask_mode=0)
    sem.sem_pmg_vcycle(P, u, out(nU))
    sem.sem_pmg_pcg_solve(P, u, out(nU), tol=1e-8)
    P.destroy()
    sem.sem_render_slice(gm, u, 2, 0.3, 31, 17, -1.0, 1.0, (0.0,), out(31 * 17, torch.float32),
                         out(31 * 17 * 4, torch.uint8))
    ta = sem.sem_tadv_create(gm, 0.01, 0.01)
    vel = [u, u, u]
    T1, N1 = out(nU), out(nL)
    sem.sem_tadv_step(ta, 0, vel, u, None, None, T1, N1)
    g0, g1 = out(nU, fill=torch.zeros(nU, dtype=f64)), out(nU, fill=torch.zeros(nU, dtype=f64))
    sem.sem_tadv_adjoint_step(ta, 1, vel, vel, u, g1, g0)
    sem.sem_tadv_nusselt_grad(ta, out(nU))
    ta.destroy()
    st = sem.sem_rbc_create(gm, 1e6, 1.0, 1e-3)
    nb = sem.sem_rbc_state_bytes(st)
    sem.sem_rbc_save_state(st, out(nb, torch.uint8))
    st.destroy()
    for k, (raw, n, dtype) in enumerate(checks):
        assert canaries_intact(raw, n, dtype), k
    gm.destroy()


def test_non_spd_helmholtz_is_rejected():
    gm = sem.sem_mesh_create_box((2, 2, 2), 3)
    b = torch.ones(gm.n_unique, dtype=torch.float64, device="cuda")
    for h1, h2 in ((1.0, -1.0), (-1.0, 0.0), (float("nan"), 1.0)):
        with pytest.raises(sem.SemError) as ei:
            sem.sem_pcg_solve(gm, h1, h2, b, torch.empty_like(b))
        assert ei.value.code == sem.SEM_ERR_INVALID_ARG
    gm.destroy()


def test_truncated_checkpoint_is_rejected(tmp_path):
    gm = sem.sem_mesh_create_box((3, 3, 3), 4, periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), deterministic=True)
    st = sem.sem_rbc_create(gm, 1e6, 1.0, 1e-3, T_pert=torch.from_numpy(
        workloads.perturbation(gm.n_unique, 1e-2, seed=2)).cuda())
    sem.sem_bdf_ext_step(st)
    path = tmp_path / "c.ckpt"
    sem.sem_rbc_save(st, str(path))
    before = sem.sem_rbc_fields(st)["T"].cpu().numpy()
    data = path.read_bytes()
    for cut in (10, 72, len(data) // 2, len(data) - 1):
        p = tmp_path / f"cut{cut}.ckpt"
        p.write_bytes(data[:cut])
        with pytest.raises(sem.SemError) as ei:
            sem.sem_rbc_load(st, str(p))
        assert ei.value.code == sem.SEM_ERR_IO
    assert np.array_equal(sem.sem_rbc_fields(st)["T"].cpu().numpy(), before)
    sem.sem_rbc_load(st, str(path))  # the whole file still loads
    st.destroy()
    gm.destroy()


def test_pcg_wall_clock_limit_returns_timeout():
    """The host-side wall-clock limit of sem_pcg_solve (opts.timeout_s): a
    solve needing thousands of iterations, given a microsecond, stops at the
    host's next check of the scalars with SEM_ERR_TIMEOUT and the iterate
    reached so far (already scaled back): CG lowers the energy
    1/2 x.Ax - b.x monotonically from its value 0 at x = 0."""
    kappa = np.array([[1.0, 2.0, 1.0], [2.0, 1.0, 1.0], [1.0, 1.0, 2.0]])
    gm = sem.sem_mesh_create_box((12, 12, 12), 7, deform_amp=0.05, kappa=kappa, phi=np.array([0.3, 1.7, 4.1]))
    _, mask = gm.maps()
    rng = np.random.default_rng(11)
    b = torch.from_numpy(rng.standard_normal(gm.n_unique) * mask).cuda()
    x = torch.zeros_like(b)
    st = sem.sem_pcg_solve(gm, 1.0, 0.0, b, x, tol=1e-14, maxit=100000, precision=sem.SEM_PREC_DF64,
                           timeout_s=1e-6, raise_on_error=False)
    assert st["status"] == sem.SEM_ERR_TIMEOUT, st
    assert 0 < st["iterations"] < 100000 and np.isfinite(st["rel_residual"])
    w = torch.zeros_like(b)
    sem.sem_ax_assembled(gm, 1.0, 0.0, x, w, sem.SEM_PREC_DF64)
    xs, ws, bs = x.cpu().numpy(), w.cpu().numpy(), b.cpu().numpy()
    assert 0.5 * xs @ ws - bs @ xs < 0.0
    gm.destroy()


def test_grid_barrier_wait_limit_ends_the_coarse_solve():
    """The grid barriers of the cooperative N = 1 coarse solve are bounded
    waits: with the bound set to one poll, CTAs that arrive early give up, the
    kernel ends without hanging and the V-cycle returns SEM_ERR_CUDA; with the
    default bound restored, the same context runs the V-cycle again and gives
    the result of an undisturbed run."""
    gm = sem.sem_mesh_create_box((24, 24, 24), 7)  # coarse level: 25^3 nodes, dozens of CTAs
    gp = sem.sem_pmg_create(gm, orders=(7, 3, 1))
    _, mask = gm.maps()
    r = torch.from_numpy(np.random.default_rng(12).standard_normal(gm.n_unique) * mask).cuda()
    z_ref = torch.zeros_like(r)
    sem.sem_pmg_vcycle(gp, r, z_ref)
    prev = sem.sem_set_grid_wait_limit(1)
    try:
        with pytest.raises(sem.SemError) as ei:
            sem.sem_pmg_vcycle(gp, r, torch.zeros_like(r))
        assert ei.value.code == sem.SEM_ERR_CUDA
        assert "grid barrier" in str(ei.value)
    finally:
        sem.sem_set_grid_wait_limit(0)
    assert prev == 1 << 24
    z = torch.zeros_like(r)
    sem.sem_pmg_vcycle(gp, r, z)
    zr = z_ref.cpu().numpy()
    assert np.abs(z.cpu().numpy() - zr).max() <= 1e-5 * np.abs(zr).max()
    gp.destroy()
    gm.destroy()
