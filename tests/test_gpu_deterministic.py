"""Deterministic assembly: with the mesh switch on, the assembled operators
sum each unique node's element contributions in ascending copy order, so
operator applications and whole solves repeat bit for bit; the results stay
within rounding of the atomic (default) mode and of the oracle's Q^T A_L Q
(Sec. 2.2)."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
import paper_2501_13240_gb300 as sem  # noqa: E402

pytestmark = pytest.mark.gpu

SPECS = [((3, 4, 5), 5, dict(deform_amp=0.05)), ((4, 3, 3), 7, dict(periodic=(1, 0, 1), dirichlet=(0, 0, 1, 1, 0, 0))),
         ((5, 2, 3), 2, dict())]


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_err(a, b):
    s = np.abs(b).max()
    return np.abs(np.asarray(a) - b).max() / (s if s > 0 else 1.0)


@pytest.mark.parametrize("prec", [sem.SEM_PREC_FP64, sem.SEM_PREC_DF64], ids=["fp64", "df64"])
@pytest.mark.parametrize("spec", SPECS, ids=["deformed_N5", "periodic_N7", "N2"])
def test_assembled_operator_is_reproducible(spec, prec):
    nel, N, kw = spec
    om = oracle.box_mesh(nel, N, **kw)
    gm = sem.sem_mesh_create_box(nel, N, **kw)
    u = torch.from_numpy(workloads.unique_field(om.n_unique, seed=5)).cuda()
    w_atomic = torch.zeros_like(u)
    sem.sem_ax_assembled(gm, 1.3, 0.7, u, w_atomic, precision=prec)
    sem.sem_mesh_set_deterministic(gm, True)
    outs = []
    for _ in range(3):
        w = torch.zeros_like(u)
        sem.sem_ax_assembled(gm, 1.3, 0.7, u, w, precision=prec)
        outs.append(host(w))
    ref = oracle.apply_assembled(om, host(u), 1.3, 0.7)
    assert rel_err(outs[0], ref) < 1e-12
    assert rel_err(outs[0], host(w_atomic)) < 1e-13
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    # the add form accumulates onto w in the same fixed order
    w = torch.from_numpy(outs[0]).cuda()
    sem.sem_ax_assembled_add(gm, 1.3, 0.7, u, w, precision=prec)
    assert rel_err(host(w), 2 * ref) < 1e-12
    sem.sem_mesh_set_deterministic(gm, False)
    gm.destroy()


@pytest.mark.parametrize("prec", [sem.SEM_PREC_FP64, sem.SEM_PREC_DF64], ids=["fp64", "df64"])
def test_pcg_solve_is_reproducible(prec):
    gm = sem.sem_mesh_create_box((5, 5, 5), 6, deform_amp=0.05, deterministic=True)
    b = torch.from_numpy(workloads.unique_field(gm.n_unique, seed=1) * gm.maps()[1]).cuda()
    xs, its = [], []
    for _ in range(2):
        x = torch.empty_like(b)
        st = sem.sem_pcg_solve(gm, 1.0, 0.1, b, x, tol=1e-10, maxit=2000, precision=prec)
        xs.append(host(x))
        its.append(st["iterations"])
    assert its[0] == its[1]
    assert np.array_equal(xs[0], xs[1])
    gm.destroy()


@pytest.mark.parametrize("gprec", [sem.SEM_PREC_FP32, sem.SEM_PREC_BF16], ids=["fp32", "bf16"])
def test_pmg_solve_is_reproducible(gprec):
    gm = sem.sem_mesh_create_box((6, 6, 6), 7, deform_amp=0.05, deterministic=True)
    P = sem.sem_pmg_create(gm, orders=(7, 3, 1), smoother_precision=gprec, coarse_tol=1e-2)
    b = torch.from_numpy(workloads.unique_field(gm.n_unique, seed=3) * gm.maps()[1]).cuda()
    xs, its = [], []
    for _ in range(2):
        x = torch.empty_like(b)
        st = sem.sem_pmg_pcg_solve(P, b, x, tol=1e-9)
        xs.append(host(x))
        its.append(st["iterations"])
    assert its[0] == its[1] and its[0] < 40
    assert np.array_equal(xs[0], xs[1])
    # same answer as the atomic hierarchy to the solve tolerance
    gm2 = sem.sem_mesh_create_box((6, 6, 6), 7, deform_amp=0.05)
    P2 = sem.sem_pmg_create(gm2, orders=(7, 3, 1), smoother_precision=gprec, coarse_tol=1e-2)
    x2 = torch.empty_like(b)
    sem.sem_pmg_pcg_solve(P2, b, x2, tol=1e-9)
    assert rel_err(host(x2), xs[0]) < 1e-6
    P2.destroy()
    gm2.destroy()
    P.destroy()
    gm.destroy()
