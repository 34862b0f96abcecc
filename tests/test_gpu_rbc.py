"""GPU parity of the BDF2/EXT2 Rayleigh-Benard step (Sec. 4.1, Eqs. (1)-(3);
Sec. 4.4 plates and periodicity) against the oracle's identical scheme, on
seeded perturbed initial states, through the C ABI."""
import numpy as np
import pytest

import oracle
from oracle import rbc
import workloads

torch = pytest.importorskip("torch")
import paper_2501_13240_gb300 as sem  # noqa: E402

pytestmark = pytest.mark.gpu


def rel_err(a, b):
    s = np.abs(b).max()
    return np.abs(np.asarray(a) - b).max() / (s if s > 0 else 1.0)


def meshes(nel, N, stretch):
    kw = dict(periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), z_stretch=stretch)
    return oracle.box_mesh(nel, N, **kw), sem.sem_mesh_create_box(nel, N, **kw)


def fields(st):
    f = sem.sem_rbc_fields(st)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in f.items()}


@pytest.mark.parametrize("pmg", [False, True], ids=["jacobi_p", "pmg_p"])
def test_conduction_state_fixed_point_gpu(pmg):
    om, gm = meshes((3, 3, 3), 5, 2.0)
    st = sem.sem_rbc_create(gm, 1e8, 0.7, 1e-3, tol=1e-12, pressure_pmg=pmg)
    z = np.zeros(om.n_unique)
    z[om.l2g] = om.Z
    pex = z - z * z / 2
    pex -= pex.mean()
    for _ in range(3):
        s = sem.sem_bdf_ext_step(st)
        f = fields(st)
        assert np.abs(f["T"] - (1.0 - z)).max() < 1e-12
        assert max(np.abs(f[c]).max() for c in "uvw") < 1e-12
        assert np.abs(f["p"] - pex).max() < 1e-10
    assert s["step"] == 3
    st.destroy()
    gm.destroy()


@pytest.mark.parametrize("pmg", [False, True], ids=["jacobi_p", "pmg_p"])
@pytest.mark.parametrize("prec", [sem.SEM_PREC_FP64, sem.SEM_PREC_DF64], ids=["fp64", "df64"])
@pytest.mark.parametrize("nel,N,stretch", [((3, 3, 3), 5, 2.0), ((2, 3, 4), 7, 1.3)])
def test_perturbed_steps_match_oracle(nel, N, stretch, prec, pmg):
    om, gm = meshes(nel, N, stretch)
    Ra, Pr, dt, tol = 1e5, 0.7, 2e-3, 1e-12
    pert = workloads.perturbation(om.n_unique, 1e-2, seed=2)
    R = rbc.RBC(om, Ra, Pr, dt, tol=tol)
    s = R.initial_state(pert)
    st = sem.sem_rbc_create(gm, Ra, Pr, dt, tol=tol, precision=prec, T_pert=torch.from_numpy(pert).cuda(),
                            pressure_pmg=pmg)
    for k in range(4):
        s = R.step(s)
        g = sem.sem_bdf_ext_step(st)
        assert g["status"] == 0
        assert abs(g["iters_T"] - s.iters["T"]) <= 2, (g, s.iters)
        if not pmg:
            assert abs(g["iters_p"] - s.iters["p"]) <= 3, (g, s.iters)
        else:
            assert g["iters_p"] * 3 < s.iters["p"], (g, s.iters)
        f = fields(st)
        assert rel_err(f["T"], s.T) < 1e-10
        assert rel_err(f["p"], s.p) < 1e-8, k
        for c, name in enumerate("uvw"):
            assert rel_err(f[name], s.u[c]) < 1e-8, (k, name)
    st.destroy()
    gm.destroy()


@pytest.mark.parametrize("order", [1, 2], ids=["ext2", "ext3"])
@pytest.mark.parametrize("pmg", [False, True], ids=["jacobi_p", "pmg_p"])
@pytest.mark.parametrize("prec", [sem.SEM_PREC_FP64, sem.SEM_PREC_DF64], ids=["fp64", "df64"])
def test_extrapolated_initial_guess_matches_oracle(prec, pmg, order):
    """Every step after the first starts its five solves from 2 x^n - x^{n-1}
    (T - Tb, p, u, v, w), and with order 2 the temperature and velocity from
    3 x^n - 3 x^{n-1} + x^{n-2} from the third step, as the oracle's option:
    four steps, same fields (T 1e-10, p and u 1e-8) and iteration counts;
    from the second step on the solves need fewer iterations than from zero."""
    om, gm = meshes((2, 3, 4), 7, 1.3)
    Ra, Pr, dt, tol = 1e5, 0.7, 2e-3, 1e-12
    pert = workloads.perturbation(om.n_unique, 1e-2, seed=2)
    R = rbc.RBC(om, Ra, Pr, dt, tol=tol, extrapolate=order)
    s = R.initial_state(pert)
    mk = dict(tol=tol, precision=prec, T_pert=torch.from_numpy(pert).cuda(), pressure_pmg=pmg)
    st = sem.sem_rbc_create(gm, Ra, Pr, dt, extrapolate=order, **mk)
    cold = sem.sem_rbc_create(gm, Ra, Pr, dt, **mk)
    for k in range(4):
        s = R.step(s)
        g = sem.sem_bdf_ext_step(st)
        c = sem.sem_bdf_ext_step(cold)
        assert g["status"] == 0 and c["status"] == 0
        assert abs(g["iters_T"] - s.iters["T"]) <= 2, (k, g, s.iters)
        if not pmg:
            assert abs(g["iters_p"] - s.iters["p"]) <= 3, (k, g, s.iters)
        for i in range(3):
            assert abs(g["iters_u"][i] - s.iters["u"][i]) <= 2, (k, g, s.iters)
        if k >= 1:
            assert g["iters_T"] < c["iters_T"] and sum(g["iters_u"]) < sum(c["iters_u"]), (k, g, c)
            assert g["iters_p"] <= c["iters_p"], (k, g, c)
        f = fields(st)
        assert rel_err(f["T"], s.T) < 1e-10, k
        assert rel_err(f["p"], s.p) < 1e-8, k
        for c_, name in enumerate("uvw"):
            assert rel_err(f[name], s.u[c_]) < 1e-8, (k, name)
    st.destroy()
    cold.destroy()
    gm.destroy()


@pytest.mark.parametrize("order", [1, 2], ids=["ext2", "ext3"])
def test_extrapolated_restart_is_bit_identical(order, tmp_path):
    """A snapshot holds p^{n-1} (and with order 2 u^{n-2}, T^{n-2}) too:
    restoring it and stepping again repeats the extrapolated run bit for bit
    (deterministic assembly); a snapshot of the other order is refused."""
    kw = dict(periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), z_stretch=1.5)
    gm = sem.sem_mesh_create_box((3, 3, 3), 5, deterministic=True, **kw)
    pert = workloads.perturbation(gm.n_unique, 1e-2, seed=2)
    st = sem.sem_rbc_create(gm, 1e7, 1.0, 2e-3, tol=1e-10, T_pert=torch.from_numpy(pert).cuda(), extrapolate=order)
    for _ in range(3):
        sem.sem_bdf_ext_step(st)
    buf = sem.sem_rbc_save_state(st)
    for _ in range(2):
        sem.sem_bdf_ext_step(st)
    ref = fields(st)
    path = str(tmp_path / "rbc.chk")
    sem.sem_rbc_save(st, path)
    other = sem.sem_rbc_create(gm, 1e7, 1.0, 2e-3, tol=1e-10, extrapolate=3 - order)
    with pytest.raises(sem.SemError):
        sem.sem_rbc_load(other, path)
    other.destroy()
    st2 = sem.sem_rbc_create(gm, 1e7, 1.0, 2e-3, tol=1e-10, extrapolate=order)
    sem.sem_rbc_load_state(st2, buf)
    for _ in range(2):
        g = sem.sem_bdf_ext_step(st2)
    assert g["step"] == 5
    again = fields(st2)
    for k in ref:
        assert np.array_equal(again[k], ref[k]), k
    st.destroy()
    st2.destroy()
    gm.destroy()


def test_rbc_mesh_requirements():
    gm = sem.sem_mesh_create_box((2, 2, 2), 3)  # walls everywhere but no periodicity: allowed
    st = sem.sem_rbc_create(gm, 1e6, 1.0, 1e-3)
    st.destroy()
    for bad in (-1, 3):  # extrapolation orders other than 0, 1, 2
        with pytest.raises(sem.SemError) as ei:
            sem.sem_rbc_create(gm, 1e6, 1.0, 1e-3, extrapolate=bad)
        assert ei.value.code == sem.SEM_ERR_INVALID_ARG
    gm.destroy()
    gm = sem.sem_mesh_create_box((2, 2, 2), 3, periodic=(1, 1, 1), dirichlet=(0,) * 6)
    with pytest.raises(sem.SemError) as ei:
        sem.sem_rbc_create(gm, 1e6, 1.0, 1e-3)
    assert ei.value.code == sem.SEM_ERR_INVALID_ARG
    gm.destroy()


def test_rbc_32_workload_step():
    """One step of the 32^3-element, N = 7 tanh-stretched RBC workload
    (Ra = 1e8, Pr = 0.7, dt = 1e-3, seeded 1e-3 perturbation)."""
    w = workloads.RBC_32
    gm = sem.mesh_from_workload(w)
    pert = workloads.perturbation(gm.n_unique, 1e-3, seed=2)
    st = sem.sem_rbc_create(gm, 1e8, 0.7, 1e-3, tol=1e-8, T_pert=torch.from_numpy(pert).cuda())
    for _ in range(2):
        g = sem.sem_bdf_ext_step(st)
        assert g["status"] == 0, g
    f = sem.sem_rbc_fields(st)
    T = f["T"]
    assert torch.isfinite(T).all() and float(T.min()) > -0.01 and float(T.max()) < 1.01
    for c in "uvw":
        assert torch.isfinite(f[c]).all()
    st.destroy()
    gm.destroy()


def test_rbc_32_workload_properties():
    """Full-size properties of the 32^3-element stretched RBC workload: with
    no perturbation the conduction state is a fixed point of the step; with
    the seeded perturbation the velocity vanishes on the plates, the pressure
    has zero mean and every field stays finite."""
    w = workloads.RBC_32
    gm = sem.mesh_from_workload(w)
    st = sem.sem_rbc_create(gm, 1e8, 0.7, 1e-3, tol=1e-10)
    for _ in range(2):
        assert sem.sem_bdf_ext_step(st)["status"] == 0
    f = sem.sem_rbc_fields(st)
    l2g, mask = gm.maps()
    Z = gm.field("Z").cpu().numpy()
    z = np.zeros(gm.n_unique)
    z[l2g] = Z
    assert np.abs(f["T"].cpu().numpy() - (1.0 - z)).max() < 1e-10
    assert max(float(f[c].abs().max()) for c in "uvw") < 1e-10
    st.destroy()
    pert = workloads.perturbation(gm.n_unique, 1e-3, seed=2)
    st = sem.sem_rbc_create(gm, 1e8, 0.7, 1e-3, tol=1e-10, T_pert=torch.from_numpy(pert).cuda())
    for _ in range(3):
        assert sem.sem_bdf_ext_step(st)["status"] == 0
    f = sem.sem_rbc_fields(st)
    walls = mask == 0
    for c in "uvw":
        assert float(f[c].cpu().numpy()[walls].__abs__().max()) == 0.0
    p = f["p"].cpu().numpy()
    assert abs(p.mean()) < 1e-12 * max(1.0, np.abs(p).max())
    for name in ("u", "v", "w", "T", "p"):
        assert torch.isfinite(f[name]).all(), name
    assert float(f["w"].abs().max()) > 0.0  # the perturbation has set the fluid moving
    st.destroy()
    gm.destroy()
