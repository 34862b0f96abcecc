"""The assembled operator on host vectors with pipelined transfers: equal to
the device-resident operator (and the oracle's Q^T A_L Q, Sec. 2.2) for
slab counts that split the lattice planes differently, periodic and
non-periodic z, N = 1 and deterministic meshes (one slab), pinned and
pageable host memory, and the full 64^3 workload; the batched form (several
applications pipelined across each other) equal to the same applications
done one by one."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
import paper_2501_13240_gb300 as sem  # noqa: E402

pytestmark = pytest.mark.gpu


def rel_err(a, b):
    s = np.abs(b).max()
    return np.abs(np.asarray(a) - b).max() / (s if s > 0 else 1.0)


SPECS = [
    (dict(nel=(5, 4, 7), N=5, deform_amp=0.05), (0, 3, 1, 7, 20)),
    (dict(nel=(3, 3, 6), N=4, periodic=(1, 1, 1), dirichlet=(0,) * 6), (4, 6, 1)),
    (dict(nel=(4, 3, 5), N=7, periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), z_stretch=2.0), (5, 2)),
    (dict(nel=(6, 5, 4), N=1, deform_amp=0.05), (4,)),
]


@pytest.mark.parametrize("prec", [sem.SEM_PREC_FP64, sem.SEM_PREC_DF64], ids=["fp64", "df64"])
@pytest.mark.parametrize("spec,chunks", SPECS, ids=["deformed_N5", "periodic_N4", "rbc_like_N7", "N1"])
def test_host_operator_matches_device_and_oracle(spec, chunks, prec):
    om = oracle.box_mesh(**spec)
    gm = sem.sem_mesh_create_box(**spec)
    u = workloads.unique_field(gm.n_unique, seed=4)
    ud = torch.from_numpy(u).cuda()
    wd = torch.empty_like(ud)
    sem.sem_ax_assembled(gm, 0.9, 2.5, ud, wd, precision=prec)
    ref_dev = wd.cpu().numpy()
    ref = oracle.apply_assembled(om, u, 0.9, 2.5)
    assert rel_err(ref_dev, ref) < 1e-12
    for nc in chunks:
        for pinned in (True, False):
            uh = torch.from_numpy(u.copy())
            wh = torch.full((gm.n_unique,), np.nan, dtype=torch.float64)
            if pinned:
                uh, wh = uh.pin_memory(), wh.pin_memory()
            sem.sem_ax_assembled_host(gm, 0.9, 2.5, uh, wh, torch.empty_like(ud), torch.empty_like(ud), prec, nc)
            got = wh.numpy()
            assert np.isfinite(got).all()
            assert rel_err(got, ref_dev) < 1e-14, (nc, pinned)
    gm.destroy()


def test_deterministic_mesh_is_bitwise_equal():
    spec = SPECS[0][0]
    gm = sem.sem_mesh_create_box(**spec, deterministic=True)
    u = workloads.unique_field(gm.n_unique, seed=4)
    ud = torch.from_numpy(u).cuda()
    wd = torch.empty_like(ud)
    sem.sem_ax_assembled(gm, 1.0, 0.0, ud, wd, precision=sem.SEM_PREC_DF64)
    wh = torch.empty(gm.n_unique, dtype=torch.float64).pin_memory()
    sem.sem_ax_assembled_host(gm, 1.0, 0.0, torch.from_numpy(u).pin_memory(), wh, torch.empty_like(ud),
                              torch.empty_like(ud), sem.SEM_PREC_DF64, 8)
    assert np.array_equal(wh.numpy(), wd.cpu().numpy())
    gm.destroy()


def test_invalid_arguments():
    gm = sem.sem_mesh_create_box((2, 2, 2), 3)
    u = torch.zeros(gm.n_unique, dtype=torch.float64)
    d = torch.zeros(gm.n_unique, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError):
        sem.sem_ax_assembled_host(gm, 1.0, 0.0, u, u.clone(), d, d, sem.SEM_PREC_DF64)  # overlapping scratch
    with pytest.raises(sem.SemError):
        sem.sem_ax_assembled_host(gm, 1.0, 0.0, u, u.clone(), d, d.clone(), 7)
    with pytest.raises(TypeError):
        sem.sem_ax_assembled_host(gm, 1.0, 0.0, u.cuda(), u.clone(), d, d.clone())
    gm.destroy()


def test_ax_gs_64_host_pipeline():
    w = workloads.AX_GS_64
    gm = sem.mesh_from_workload(w)
    u = workloads.unique_field(gm.n_unique, seed=0)
    ud = torch.from_numpy(u).cuda()
    wd = torch.empty_like(ud)
    sem.sem_ax_assembled(gm, 1.0, 0.0, ud, wd, precision=sem.SEM_PREC_DF64)
    uh = torch.from_numpy(u).pin_memory()
    wh = torch.empty(gm.n_unique, dtype=torch.float64).pin_memory()
    sem.sem_ax_assembled_host(gm, 1.0, 0.0, uh, wh, torch.empty_like(ud), torch.empty_like(ud))
    assert rel_err(wh.numpy(), wd.cpu().numpy()) < 1e-14
    gm.destroy()


@pytest.mark.parametrize("prec", [sem.SEM_PREC_FP64, sem.SEM_PREC_DF64], ids=["fp64", "df64"])
@pytest.mark.parametrize("si", [0, 2, 3], ids=["deformed_N5", "rbc_like_N7", "N1"])
def test_host_batch_matches_device_and_oracle(si, prec):
    spec = SPECS[si][0]
    om = oracle.box_mesh(**spec)
    gm = sem.sem_mesh_create_box(**spec)
    K = 5
    us = [workloads.unique_field(gm.n_unique, seed=10 + k) for k in range(K)]
    u_hosts = [torch.from_numpy(u.copy()).pin_memory() for u in us]
    w_hosts = [torch.full((gm.n_unique,), np.nan, dtype=torch.float64).pin_memory() for _ in range(K)]
    u2 = torch.empty(2 * gm.n_unique, dtype=torch.float64, device="cuda")
    w2 = torch.empty_like(u2)
    sem.sem_ax_assembled_host_batch(gm, 0.9, 2.5, u_hosts, w_hosts, u2, w2, prec)
    wd = torch.empty(gm.n_unique, dtype=torch.float64, device="cuda")
    for k in range(K):
        sem.sem_ax_assembled(gm, 0.9, 2.5, torch.from_numpy(us[k]).cuda(), wd, precision=prec)
        got = w_hosts[k].numpy()
        assert np.isfinite(got).all()
        assert rel_err(got, wd.cpu().numpy()) < 1e-14, k
        assert rel_err(got, oracle.apply_assembled(om, us[k], 0.9, 2.5)) < 1e-12, k
    gm.destroy()


def test_host_batch_shared_buffers_and_edge_cases():
    spec = SPECS[0][0]
    gm = sem.sem_mesh_create_box(**spec, deterministic=True)
    u = workloads.unique_field(gm.n_unique, seed=4)
    ud = torch.from_numpy(u).cuda()
    wd = torch.empty_like(ud)
    sem.sem_ax_assembled(gm, 1.0, 0.0, ud, wd, precision=sem.SEM_PREC_DF64)
    ref = wd.cpu().numpy()
    # one input read by every application, two output buffers written alternately
    uh = torch.from_numpy(u).pin_memory()
    outs = [torch.full((gm.n_unique,), np.nan, dtype=torch.float64).pin_memory() for _ in range(2)]
    u2 = torch.empty(2 * gm.n_unique, dtype=torch.float64, device="cuda")
    w2 = torch.empty_like(u2)
    sem.sem_ax_assembled_host_batch(gm, 1.0, 0.0, [uh] * 7, [outs[k % 2] for k in range(7)], u2, w2)
    for o in outs:  # deterministic mesh: bit for bit the device-resident result
        assert np.array_equal(o.numpy(), ref)
    # no applications: nothing happens
    o = torch.full((gm.n_unique,), 7.0, dtype=torch.float64)
    sem.sem_ax_assembled_host_batch(gm, 1.0, 0.0, [], [], u2, w2)
    assert (o.numpy() == 7.0).all()
    with pytest.raises(sem.SemError):  # identical device buffers
        sem.sem_ax_assembled_host_batch(gm, 1.0, 0.0, [uh], [o], u2, u2)
    with pytest.raises(sem.SemError):  # unknown precision
        sem.sem_ax_assembled_host_batch(gm, 1.0, 0.0, [uh], [o], u2, w2, 7)
    with pytest.raises(ValueError):
        sem.sem_ax_assembled_host_batch(gm, 1.0, 0.0, [uh, uh], [o], u2, w2)
    gm.destroy()
