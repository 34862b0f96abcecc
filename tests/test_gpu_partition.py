"""The GPU half of the element-slab partition (Sec. 2.2: one rank per GPU,
shared surface values summed across ranks, the exchange overlapped with the
interior elements), through the C ABI against the FP64 oracle:

* the element-list operator against the oracle's sum over the same elements;
* each rank's slab mesh (its own numbering) against the oracle's partial
  sums over the rank's elements, in one process;
* the overlapped schedule (surface elements, host exchange, interior
  elements on a second stream) and the partitioned Jacobi-PCG on 2 and 3
  processes sharing the GPU, exchanging through gloo host buffers: the
  assembled result equals the oracle's Q Q^T A_L to 1e-12 and the solve
  equals the single-partition solve (iterations +-1, x to 1e-9).

The ranks' kernels never wait on one another: every exchange is on the host.
"""
import os
import socket

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import paper_2501_13240_gb300 as sem  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KAPPA = np.array([[1.0, 2.0, 1.0], [2.0, 1.0, 1.0], [1.0, 1.0, 2.0]])
PHI = np.array([0.3, 1.7, 4.1])

CASES = [dict(nel=(3, 2, 4), N=7, periodic=(0, 0, 0), dirichlet=(1,) * 6, deform_amp=0.05),
         dict(nel=(2, 3, 6), N=4, periodic=(1, 1, 1), dirichlet=(0,) * 6, deform_amp=0.0),
         dict(nel=(2, 2, 5), N=7, periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), deform_amp=0.04, z_stretch=1.5)]


def _box(case):
    kw = dict(periodic=case["periodic"], dirichlet=case["dirichlet"], deform_amp=case["deform_amp"],
              z_stretch=case.get("z_stretch", 0.0), kappa=KAPPA, phi=PHI)
    om = oracle.box_mesh(case["nel"], case["N"], **kw)
    desc = sem.box_desc(case["nel"], case["N"], **kw)
    return om, desc, kw


def rel_err(a, b):
    s = np.abs(b).max()
    return np.abs(np.asarray(a) - b).max() / (s if s > 0 else 1.0)


def _oracle_elems(om, ug, elems, h1, h2):
    """sum over the listed elements of Q_e^T A_e Q_e (masked), unique-node vector"""
    n3 = (om.N + 1) ** 3
    idx = (np.asarray(elems)[:, None] * n3 + np.arange(n3)[None, :]).ravel()
    uL = (ug * om.mask)[om.l2g[idx]]
    wl = oracle.ax_local_raw(om.N, om.D, np.ascontiguousarray(om.G[:, idx]), np.ascontiguousarray(om.B[idx]), uL,
                             h1, h2)
    out = np.zeros(om.n_unique)
    np.add.at(out, om.l2g[idx], wl)
    return out * om.mask


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec", [sem.SEM_PREC_DF64, sem.SEM_PREC_FP64], ids=["df64", "fp64"])
def test_element_list_operator(case, prec):
    om, desc, kw = _box(CASES[case])
    gm = sem.sem_mesh_create_box(CASES[case]["nel"], CASES[case]["N"], **kw)
    rng = np.random.default_rng(40 + case)
    ug = rng.uniform(-1, 1, om.n_unique)
    for elems in (np.arange(om.E), rng.choice(om.E, size=max(1, om.E // 3), replace=False), np.array([om.E - 1])):
        w = torch.zeros(om.n_unique, dtype=torch.float64, device="cuda")
        el = torch.from_numpy(elems.astype(np.int32)).cuda()
        sem.sem_ax_assembled_elems(gm, 0.4, 7.0, torch.from_numpy(ug).cuda(), w, el, precision=prec)
        ref = _oracle_elems(om, ug, elems, 0.4, 7.0)
        assert rel_err(w.cpu().numpy(), ref) < 1e-12
    # a list longer than the mesh is rejected
    with pytest.raises(sem.SemError):
        big = torch.zeros(om.E + 1, dtype=torch.int32, device="cuda")
        sem.sem_ax_assembled_elems(gm, 1.0, 0.0, torch.from_numpy(ug).cuda(), w, big)
    gm.destroy()


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("world", [1, 2, 3])
def test_slab_meshes_hold_the_ranks_partial_sums(case, world):
    """In one process: every rank's slab mesh (geometry, its own numbering,
    Dirichlet faces) applies the operator over the rank's elements; mapped to
    the box's ids it equals the oracle's partial sums over those elements."""
    om, desc, kw = _box(CASES[case])
    ug = np.random.default_rng(50 + case).uniform(-1, 1, om.n_unique)
    for rank in range(world):
        P = sem.sem_part_create(desc, world, rank)
        gid = P.global_ids()
        assert len(np.unique(gid)) == P.n_unique
        _, mask = P.mesh.maps()
        np.testing.assert_array_equal(mask, om.mask[gid])
        u = torch.from_numpy(ug[gid]).cuda()
        w = torch.zeros_like(u)
        sem.sem_ax_assembled(P.mesh, 0.4, 7.0, u, w, sem.SEM_PREC_DF64)
        ref = _oracle_elems(om, ug, np.arange(P.e_begin, P.e_end), 0.4, 7.0)
        assert rel_err(w.cpu().numpy(), ref[gid]) < 1e-12, rank
        assert P.n_surface + P.n_interior == P.e_end - P.e_begin
        assert (P.n_interface > 0) == (world > 1)
        P.destroy()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_worker(rank, world, port, case, queue):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as orc
        import paper_2501_13240_gb300 as sm
        torch.cuda.set_device(0)
        om, desc, _ = _box(case)
        P = sm.sem_part_create(desc, world, rank)
        gid = P.global_ids()
        mine, _ = sm.sem_partition_interface(desc, world, rank)
        allg = np.unique(np.concatenate([sm.sem_partition_interface(desc, world, q)[0] for q in range(world)]))
        slot = np.searchsorted(allg, mine)
        calls = {"exchange": 0}

        def exchange(buf):  # sum over the ranks holding each interface node, via gloo
            calls["exchange"] += 1
            t = torch.zeros(len(allg), dtype=torch.float64)
            t[slot] = torch.from_numpy(buf.copy())
            dist.all_reduce(t)
            buf[:] = t.numpy()[slot]

        def allreduce(vals):
            t = torch.from_numpy(vals.copy())
            dist.all_reduce(t)
            vals[:] = t.numpy()

        res = {}
        for prec in (sm.SEM_PREC_DF64, sm.SEM_PREC_FP64):
            ug = np.random.default_rng(60).uniform(-1, 1, om.n_unique)
            u = torch.from_numpy(ug[gid]).cuda()
            w = torch.zeros_like(u)
            P.ax(0.4, 7.0, u, w, exchange, precision=prec)
            torch.cuda.synchronize()
            ref = orc.apply_assembled(om, ug, 0.4, 7.0)
            res["ax_err_%d" % prec] = float(np.abs(w.cpu().numpy() - ref[gid]).max() / np.abs(ref).max())
        res["exchanges"] = calls["exchange"]
        # partitioned Jacobi-PCG against the single-partition oracle solve
        h2 = 0.0 if case["dirichlet"][0] or case["dirichlet"][4] else 0.5
        b_all = om.mask * np.random.default_rng(61).standard_normal(om.n_unique)
        ref = orc.pcg(om, b_all, 1.0, h2, tol=1e-10, maxit=3000)
        b = torch.from_numpy(b_all[gid]).cuda()
        x = torch.zeros_like(b)
        st = P.pcg_solve(1.0, h2, b, x, exchange, allreduce, tol=1e-10, maxit=3000)
        res["its"], res["ref_its"] = st["iterations"], ref.iterations
        res["x_err"] = float(np.abs(x.cpu().numpy() - ref.x[gid]).max() / np.abs(ref.x).max())
        res["status"] = st["status"]
        P.destroy()
        queue.put((rank, res))
    except Exception as exc:  # report instead of hanging the parent
        queue.put((rank, {"error": repr(exc)}))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_overlapped_operator_and_solve_on_ranks_sharing_the_gpu(world, case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker, args=(r, world, port, CASES[case], q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=600) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank in range(world):
        r = res[rank]
        assert "error" not in r, r
        assert r["ax_err_1"] < 1e-12 and r["ax_err_0"] < 1e-12, (rank, r)
        assert r["exchanges"] == 2  # one per operator application
        assert r["status"] == 0 and abs(r["its"] - r["ref_its"]) <= 1, (rank, r)
        assert r["x_err"] < 1e-9, (rank, r)
    assert len({res[k]["its"] for k in res}) == 1  # every rank stops at the same iteration
