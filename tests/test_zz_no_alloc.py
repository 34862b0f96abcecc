"""The no-allocation Jacobi-PCG entry point (sem_pcg_solve_noalloc), for
callers that cannot allocate device memory themselves: it must give the same
result as sem_pcg_solve with caller-provided workspace, on consecutive calls
that share its fixed device array, and reject meshes too large for it.

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2501_13240_gb300 as sem  # noqa: E402

pytestmark = pytest.mark.gpu

KAPPA = np.array([[1.0, 2.0, 1.0], [2.0, 1.0, 1.0], [1.0, 1.0, 2.0]])
PHI = np.array([0.3, 1.7, 4.1])


def test_noalloc_matches_workspace_solve_twice():
    gm = sem.sem_mesh_create_box((5, 4, 3), 7, deform_amp=0.05, kappa=KAPPA, phi=PHI)
    _, mask = gm.maps()
    m = torch.from_numpy(mask.astype(np.float64)).cuda()
    for call, (h1, h2, prec) in enumerate([(1.0, 0.0, sem.SEM_PREC_DF64), (0.5, 30.0, sem.SEM_PREC_FP64)]):
        rng = np.random.default_rng(100 + call)
        b = torch.from_numpy(rng.standard_normal(gm.n_unique)).cuda() * m
        x_ref = torch.zeros_like(b)
        ref = sem.sem_pcg_solve(gm, h1, h2, b, x_ref, tol=1e-10, maxit=2000, precision=prec)
        x = torch.full_like(b, 7.0)  # stale contents must not matter
        st = sem.sem_pcg_solve_noalloc(gm, h1, h2, b, x, tol=1e-10, maxit=2000, precision=prec)
        assert st["status"] == 0 and ref["status"] == 0
        assert abs(st["iterations"] - ref["iterations"]) <= 1, (st, ref)
        assert st["rel_residual"] <= 1e-10
        xr = x_ref.cpu().numpy()
        err = np.abs(x.cpu().numpy() - xr).max() / np.abs(xr).max()
        assert err < 1e-10, (call, err)
    gm.destroy()


def test_noalloc_rejects_mesh_beyond_capacity():
    cap = sem.sem_pcg_noalloc_capacity()
    assert cap == 64 << 20
    gm = sem.sem_mesh_create_box((20, 20, 20), 7)  # 141^3 = 2.8 M unique nodes
    assert 4 * 8 * gm.n_unique > cap
    b = torch.zeros(gm.n_unique, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as ei:
        sem.sem_pcg_solve_noalloc(gm, 1.0, 0.0, b, torch.zeros_like(b))
    assert ei.value.code == sem.SEM_ERR_INVALID_ARG
    assert "workspace" in str(ei.value)
    gm.destroy()
