"""GPU parity of the frozen-velocity temperature step, its discrete adjoint and
the bottom-plate Nusselt functional (Sec. 4.1 Eq. (2); plates of Sec. 4.4)
against the oracle; RBC checkpoints (bit-identical restart); and the
checkpointed autograd gradient of Nu_b after K steps, checked by central
finite differences on seeded directions."""
import numpy as np
import pytest

import oracle
from oracle import adjoint, rbc
import workloads

torch = pytest.importorskip("torch")
import paper_2501_13240_gb300 as sem  # noqa: E402
from paper_2501_13240_gb300 import adjoint as gadj  # noqa: E402

pytestmark = pytest.mark.gpu

KW = dict(periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1))


def rel_err(a, b):
    s = np.abs(b).max()
    return np.abs(np.asarray(a) - b).max() / (s if s > 0 else 1.0)


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def velocities(m, K, amp=0.3, seed=4):
    rng = np.random.default_rng(seed)
    return [[amp * rng.standard_normal(m.n_unique) * m.mask for _ in range(3)] for _ in range(K)]


CASES = [((2, 2, 3), 4, 1.5, 0.0), ((3, 2, 2), 6, 1.0, 0.04), ((2, 3, 2), 7, 2.0, 0.0)]


@pytest.fixture(params=CASES, ids=lambda c: f"{c[0][0]}x{c[0][1]}x{c[0][2]}_N{c[1]}")
def pair(request):
    nel, N, stretch, amp = request.param
    om = oracle.box_mesh(nel, N, z_stretch=stretch, deform_amp=amp, **KW)
    gm = sem.sem_mesh_create_box(nel, N, z_stretch=stretch, deform_amp=amp, **KW)
    yield om, gm
    gm.destroy()


def test_nusselt_and_gradient_match_oracle(pair):
    om, gm = pair
    oa = adjoint.TAdv(om, 0.02, 0.005)
    ta = sem.sem_tadv_create(gm, 0.02, 0.005)
    assert abs(ta.area() - adjoint.bottom_weights(om, oa.g).sum()) < 1e-13
    assert rel_err(host(ta.lifting()), oa.Tb) == 0.0 or rel_err(host(ta.lifting()), oa.Tb) < 1e-15
    # conduction: exactly 1
    assert abs(sem.sem_tadv_nusselt(ta, ta.lifting()) - 1.0) < 1e-12
    T = np.random.default_rng(3).standard_normal(om.n_unique)
    nu = sem.sem_tadv_nusselt(ta, cuda(T))
    ref = adjoint.nusselt_bottom(om, oa.g, T)
    assert abs(nu - ref) <= 1e-12 * max(1.0, abs(ref))
    c = torch.empty(om.n_unique, dtype=torch.float64, device="cuda")
    sem.sem_tadv_nusselt_grad(ta, c, scale=-2.5)
    assert rel_err(host(c), -2.5 * adjoint.nusselt_bottom_grad(om, oa.g)) < 1e-12
    ta.destroy()


@pytest.mark.parametrize("prec", [sem.SEM_PREC_FP64, sem.SEM_PREC_DF64], ids=["fp64", "df64"])
def test_forward_steps_match_oracle(pair, prec):
    om, gm = pair
    kappa, dt, K = 0.02, 0.005, 4
    oa = adjoint.TAdv(om, kappa, dt, tol=1e-13)
    ta = sem.sem_tadv_create(gm, kappa, dt, tol=1e-13, precision=prec)
    us = velocities(om, K)
    T0 = oa.Tb + 0.1 * np.random.default_rng(2).standard_normal(om.n_unique) * oa.mk
    To, Tpo, Npo = T0, None, None
    Tg, Tpg, Npg = cuda(T0), None, None
    for n in range(K):
        To1, No = oa.step(n, us[n], To, Tpo, Npo)
        Tg1 = torch.empty_like(Tg)
        Ng = torch.empty(om.n_local, dtype=torch.float64, device="cuda")
        sem.sem_tadv_step(ta, n, [cuda(c) for c in us[n]], Tg, Tpg, Npg, Tg1, Ng)
        assert rel_err(host(Ng), No) < 1e-12, n
        assert rel_err(host(Tg1), To1) < 1e-11, n
        To, Tpo, Npo = To1, To, No
        Tg, Tpg, Npg = Tg1, Tg, Ng
    ta.destroy()


def gpu_adjoint(ta, us_g, gK):
    K = len(us_g)
    g = [torch.zeros_like(gK) for _ in range(K + 1)]
    g[K].copy_(gK)
    for n in range(K - 1, -1, -1):
        sem.sem_tadv_adjoint_step(ta, n, us_g[n], us_g[n - 1] if n > 0 else None, g[n + 1], g[n],
                                  g[n - 1] if n > 0 else None)
    return g[0]


@pytest.mark.parametrize("prec", [sem.SEM_PREC_FP64, sem.SEM_PREC_DF64], ids=["fp64", "df64"])
def test_adjoint_matches_oracle(pair, prec):
    om, gm = pair
    kappa, dt, K = 0.02, 0.005, 5
    oa = adjoint.TAdv(om, kappa, dt, tol=1e-13)
    ta = sem.sem_tadv_create(gm, kappa, dt, tol=1e-13, precision=prec)
    us = velocities(om, K, amp=0.5, seed=9)
    c = adjoint.nusselt_bottom_grad(om, oa.g)
    ref = oa.adjoint(c, us)
    got = host(gpu_adjoint(ta, [[cuda(x) for x in u] for u in us], cuda(c)))
    assert rel_err(got, ref) < 1e-11
    assert np.all(got[om.mask == 0] == 0.0)
    ta.destroy()


def test_adjoint_dot_product_identity_gpu():
    """<g0, d> = Nu(T^K(T0 + d)) - Nu(T^K(T0)) for the affine map, all on the GPU."""
    om = oracle.box_mesh((3, 3, 3), 5, z_stretch=1.5, **KW)
    gm = sem.sem_mesh_create_box((3, 3, 3), 5, z_stretch=1.5, **KW)
    ta = sem.sem_tadv_create(gm, 0.01, 0.01, tol=1e-13)
    K = 6
    us_g = [[cuda(x) for x in u] for u in velocities(om, K, amp=0.4, seed=5)]

    def run(T0):
        Tn, Tp, Np = T0, None, None
        for n in range(K):
            T1 = torch.empty_like(Tn)
            N1 = torch.empty(om.n_local, dtype=torch.float64, device="cuda")
            sem.sem_tadv_step(ta, n, us_g[n], Tn, Tp, Np, T1, N1)
            Tn, Tp, Np = T1, Tn, N1
        return sem.sem_tadv_nusselt(ta, Tn)

    c = torch.empty(om.n_unique, dtype=torch.float64, device="cuda")
    sem.sem_tadv_nusselt_grad(ta, c)
    g0 = host(gpu_adjoint(ta, us_g, c))
    T0 = host(ta.lifting())
    d = np.random.default_rng(8).standard_normal(om.n_unique) * om.mask
    dJ = run(cuda(T0 + d)) - run(cuda(T0))
    assert abs(dJ - np.dot(g0, d)) <= 1e-9 * abs(dJ), (dJ, np.dot(g0, d))
    ta.destroy()
    gm.destroy()


def test_invalid_arguments():
    gm = sem.sem_mesh_create_box((2, 2, 2), 3, **KW)
    with pytest.raises(sem.SemError):
        sem.sem_tadv_create(gm, -1.0, 0.01)
    walls = sem.sem_mesh_create_box((2, 2, 2), 3, periodic=(1, 1, 1), dirichlet=(0,) * 6)
    with pytest.raises(sem.SemError):
        sem.sem_tadv_create(walls, 0.1, 0.01)
    ta = sem.sem_tadv_create(gm, 0.1, 0.01)
    u = [torch.zeros(gm.n_unique, dtype=torch.float64, device="cuda") for _ in range(3)]
    T = torch.zeros(gm.n_unique, dtype=torch.float64, device="cuda")
    N = torch.zeros(gm.n_local, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError):  # n > 0 needs the history
        sem.sem_tadv_step(ta, 1, u, T, None, None, T.clone(), N)
    with pytest.raises(sem.SemError):
        sem.sem_tadv_adjoint_step(ta, 2, u, None, T, T.clone(), T.clone())
    ta.destroy()
    walls.destroy()
    gm.destroy()


# ------------------------------------------------------------------ checkpoints

def rbc_run(nel=(3, 3, 3), N=5, Ra=1e7, Pr=1.0, dt=2e-3, tol=1e-10):
    om = oracle.box_mesh(nel, N, z_stretch=1.5, **KW)
    gm = sem.sem_mesh_create_box(nel, N, z_stretch=1.5, deterministic=True, **KW)
    pert = workloads.perturbation(om.n_unique, 1e-2, seed=2)
    st = sem.sem_rbc_create(gm, Ra, Pr, dt, tol=tol, T_pert=cuda(pert))
    return om, gm, st, pert


def all_fields(st):
    f = sem.sem_rbc_fields(st)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in f.items()}


def test_snapshot_restart_is_bit_identical(tmp_path):
    om, gm, st, _ = rbc_run()
    for _ in range(3):
        sem.sem_bdf_ext_step(st)
    buf = sem.sem_rbc_save_state(st)
    path = str(tmp_path / "rbc.ckpt")
    sem.sem_rbc_save(st, path)
    for _ in range(2):
        sem.sem_bdf_ext_step(st)
    ref = all_fields(st)
    sem.sem_rbc_load_state(st, buf)
    assert all_fields(st)["u"].shape == ref["u"].shape
    for _ in range(2):
        sem.sem_bdf_ext_step(st)
    again = all_fields(st)
    sem.sem_rbc_load(st, path)
    assert sem.sem_rbc_fields(st)  # loads
    for _ in range(2):
        s = sem.sem_bdf_ext_step(st)
    from_file = all_fields(st)
    assert s["step"] == 5
    for k in ref:
        assert np.array_equal(again[k], ref[k]), k
        assert np.array_equal(from_file[k], ref[k]), k
    # corrupted / foreign checkpoints are rejected and leave the state alone
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0x01
    bad = str(tmp_path / "bad.ckpt")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(sem.SemError):
        sem.sem_rbc_load(st, bad)
    with pytest.raises(sem.SemError):
        sem.sem_rbc_load(st, str(tmp_path / "missing.ckpt"))
    assert np.array_equal(all_fields(st)["T"], ref["T"])
    om2 = sem.sem_mesh_create_box((2, 3, 3), 5, z_stretch=1.5, **KW)
    st2 = sem.sem_rbc_create(om2, 1e7, 1.0, 2e-3)
    with pytest.raises(sem.SemError):
        sem.sem_rbc_load(st2, path)
    st3 = sem.sem_rbc_create(gm, 1e7, 1.0, 1e-3)  # same mesh, another dt
    with pytest.raises(sem.SemError):
        sem.sem_rbc_load(st3, path)
    with pytest.raises(sem.SemError):
        sem.sem_rbc_load_state(st3, buf)
    st3.destroy()
    with pytest.raises(sem.SemError):
        sem.sem_rbc_load_state(st2, torch.zeros(sem.sem_rbc_state_bytes(st2), dtype=torch.uint8, device="cuda"))
    st2.destroy()
    om2.destroy()
    st.destroy()
    gm.destroy()


def test_history_replay_and_transport_reproduce_the_run():
    """Velocities regenerated from checkpoints equal the original run's, and the
    frozen-velocity transport from T^0 reproduces the run's own T^K."""
    om, gm, st, pert = rbc_run()
    K, every = 7, 3
    T0 = sem.sem_rbc_fields(st)["T"]
    kept = []
    ref = sem.sem_rbc_create(gm, 1e7, 1.0, 2e-3, tol=1e-10, T_pert=cuda(pert))
    for _ in range(K):
        f = all_fields(ref)
        kept.append([f["u"], f["v"], f["w"]])
        sem.sem_bdf_ext_step(ref)
    TK_run = all_fields(ref)["T"]
    hist = gadj.VelocityHistory(st, K, every)
    assert hist.n_segments == 3
    for s in range(hist.n_segments):
        vel = hist.segment(s)
        for n, u in vel.items():
            for c in range(3):
                assert np.array_equal(host(u[c]), kept[n][c]), (s, n, c)
    ta = sem.sem_tadv_create(gm, 1.0 / np.sqrt(1e7), 2e-3, tol=1e-10, precision=sem.SEM_PREC_DF64)
    TK = host(hist.transport(ta, T0))
    assert np.array_equal(TK, TK_run)
    assert all_fields(st)["T"].tobytes() == TK_run.tobytes()  # left at step K
    ta.destroy()
    ref.destroy()
    st.destroy()
    gm.destroy()


def test_autograd_gradient_small_matches_oracle_and_fd():
    om, gm, st, pert = rbc_run(nel=(2, 2, 3), N=4)
    K, every, dt = 6, 5, 2e-3
    kappa = 1.0 / np.sqrt(1e7)
    hist = gadj.VelocityHistory(st, K, every)
    us = []
    for s in range(hist.n_segments):
        vel = hist.segment(s)
        n0, n1 = hist.bounds(s)
        us += [[host(c) for c in vel[n]] for n in range(n0, n1)]
    hist.restore()
    ta = sem.sem_tadv_create(gm, kappa, dt, tol=1e-13)
    oa = adjoint.TAdv(om, kappa, dt, tol=1e-13)
    T0 = sem.sem_tadv_create(gm, kappa, dt).lifting() + cuda(pert * om.mask)
    x = T0.clone().requires_grad_(True)
    nu = gadj.nusselt_after(x, hist, ta)
    nu.backward()
    g = host(x.grad)
    ref = oa.adjoint(adjoint.nusselt_bottom_grad(om, oa.g), us)
    assert rel_err(g, ref) < 1e-10
    assert abs(float(nu.detach()) - adjoint.nusselt_bottom(om, oa.g, oa.forward(host(T0), us))) < 1e-11
    rng = np.random.default_rng(21)
    eps = 1e-6
    for _ in range(3):
        d = cuda(rng.standard_normal(om.n_unique) * om.mask)
        fd = (float(gadj.nusselt_after(T0 + eps * d, hist, ta)) - float(gadj.nusselt_after(T0 - eps * d, hist, ta))) / (2 * eps)
        gd = float(torch.dot(x.grad, d))
        assert abs(fd - gd) <= 1e-6 * abs(fd), (fd, gd)
    ta.destroy()
    st.destroy()
    gm.destroy()


@pytest.mark.slow
def test_adjoint_16_gradient_fd_ten_directions():
    """The full workload: 16^3 elements, N = 7, Ra = 1e7, Pr = 1, K = 20 steps,
    checkpoints every 5 steps; central FD with eps = 1e-6 on 10 seeded
    directions."""
    w = workloads.ADJOINT_16
    gm = sem.sem_mesh_create_box(w.nel, w.N, deterministic=True, **KW)
    Ra, Pr, dt, K = 1e7, 1.0, 2e-3, 20
    pert = workloads.perturbation(w.n_unique, 1e-2, seed=2)
    st = sem.sem_rbc_create(gm, Ra, Pr, dt, tol=1e-10, T_pert=cuda(pert))
    T0 = sem.sem_rbc_fields(st)["T"]
    hist = gadj.VelocityHistory(st, K, 5)
    assert max(s["status"] for s in hist.stats) == 0
    ta = sem.sem_tadv_create(gm, 1.0 / np.sqrt(Ra * Pr), dt, tol=1e-13, precision=sem.SEM_PREC_DF64)
    x = T0.clone().requires_grad_(True)
    nu = gadj.nusselt_after(x, hist, ta)
    nu.backward()
    assert 0.5 < float(nu.detach()) < 5.0
    mask = cuda(gm.maps()[1].astype(np.float64))
    rng = np.random.default_rng(31)
    eps = 1e-6
    for _ in range(10):
        d = torch.from_numpy(rng.standard_normal(w.n_unique)).cuda() * mask
        fd = (float(gadj.nusselt_after(T0 + eps * d, hist, ta)) - float(gadj.nusselt_after(T0 - eps * d, hist, ta))) / (2 * eps)
        gd = float(torch.dot(x.grad, d))
        assert abs(fd - gd) <= 1e-5 * abs(fd), (fd, gd)
    ta.destroy()
    st.destroy()
    gm.destroy()
