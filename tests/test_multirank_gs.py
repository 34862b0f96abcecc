"""Multi-rank direct stiffness summation on CPU ranks (gloo): the element-slab
partition's interface maps against brute force (bit-exact), and the summed
result against the single-partition Q Q^T (Sec. 2.2: one rank per GPU,
shared surface values summed across ranks) both by an all-reduce and by
pairwise exchanges over the neighbour plan, the surface-first overlapped
schedule, and a whole Jacobi-PCG over the partition against the
single-partition solve."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [dict(nel=(3, 2, 4), N=3, periodic=(0, 0, 0), dirichlet=(1,) * 6),
         dict(nel=(2, 3, 6), N=4, periodic=(1, 1, 1), dirichlet=(0,) * 6),
         dict(nel=(2, 2, 5), N=2, periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1))]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, queue):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import paper_2501_13240_gb300 as sem
        om = oracle.box_mesh(case["nel"], case["N"], periodic=case["periodic"], dirichlet=case["dirichlet"])
        desc = sem.box_desc(case["nel"], case["N"], periodic=case["periodic"], dirichlet=case["dirichlet"])
        n3 = (case["N"] + 1) ** 3
        e0, e1, ni = sem.sem_partition_info(desc, world, rank)
        mine = slice(e0 * n3, e1 * n3)
        gids, nshare = sem.sem_partition_interface(desc, world, rank)
        # brute force: unique ids this rank holds that another rank also holds
        own = np.unique(om.l2g[mine])
        other = np.unique(np.concatenate([om.l2g[: e0 * n3], om.l2g[e1 * n3:]]))
        brute = np.intersect1d(own, other)
        maps_ok = np.array_equal(gids, brute)
        holders = np.zeros(om.n_unique, dtype=np.int32)
        for q in range(world):
            a, b, _ = sem.sem_partition_info(desc, world, q)
            holders[np.unique(om.l2g[a * n3:b * n3])] += 1
        share_ok = np.array_equal(nshare, holders[gids])
        # rank-local partial sums, then exchange of the interface partial sums
        v = np.random.default_rng(17).standard_normal(om.n_local)
        part = np.zeros(om.n_unique)
        np.add.at(part, om.l2g[mine], v[mine])
        allg = np.unique(np.concatenate([sem.sem_partition_interface(desc, world, q)[0] for q in range(world)]))
        buf = torch.zeros(len(allg), dtype=torch.float64)
        idx = np.searchsorted(allg, gids)
        buf[idx] = torch.from_numpy(part[gids])
        dist.all_reduce(buf)
        part[gids] = buf.numpy()[idx]
        got = part[om.l2g[mine]]
        ref = oracle.qqt(om, v)[mine]
        err = float(np.abs(got - ref).max() / np.abs(ref).max())
        queue.put((rank, bool(maps_ok), bool(share_ok), err, int(ni)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_partitioned_gather_scatter(world, case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, CASES[case], q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, maps_ok, share_ok, err, ni in sorted(res):
        assert maps_ok and share_ok, (rank, ni)
        assert err < 1e-14, (rank, err)
        assert ni > 0


def test_partition_rejects_bad_arguments():
    import paper_2501_13240_gb300 as sem
    d = sem.box_desc((2, 2, 2), 3)
    with pytest.raises(sem.SemError):
        sem.sem_partition_info(d, 3, 0)  # more ranks than element planes
    with pytest.raises(sem.SemError):
        sem.sem_partition_info(d, 2, 2)
    assert sem.sem_partition_info(d, 1, 0) == (0, 8, 0)


def _worker_failing(rank, world, port, queue):
    """Rank 1 fails (raises) after joining and before the interface exchange;
    rank 0 must learn of it on the host instead of hanging: first from a
    missing heartbeat in the rendezvous store, then from its exchange ending
    with an error within the process group's timeout."""
    import datetime
    import sys
    import time
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    store = dist.distributed_c10d._get_default_store()
    if rank == 1:
        queue.put((1, "failing", 0.0))
        queue.close()
        queue.join_thread()  # the message is out before the process dies
        os._exit(3)  # dies with no exchange in flight
    t0 = time.monotonic()
    heartbeat_missing = False
    try:
        store.wait(["heartbeat/1/step0"], datetime.timedelta(seconds=3))
    except Exception:
        heartbeat_missing = True
    exchange_failed = False
    try:
        buf = torch.zeros(8, dtype=torch.float64)
        dist.all_reduce(buf)
    except Exception:
        exchange_failed = True
    queue.put((0, f"heartbeat_missing={heartbeat_missing} exchange_failed={exchange_failed}",
               time.monotonic() - t0))
    queue.close()
    queue.join_thread()
    os._exit(0)  # skip the process-group teardown, which would wait for the dead peer


def test_failed_rank_is_detected_on_the_host():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_failing, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (msg, t)) for r, msg, t in (q.get(timeout=120) for _ in range(2)))
    for p in procs:
        p.join(timeout=60)
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
    msg, elapsed = res[0]
    assert msg == "heartbeat_missing=True exchange_failed=True", msg
    assert elapsed < 30.0


def _worker_pcg(rank, world, port, case, h2, queue):
    """Jacobi-PCG over the element-slab partition: each rank applies the local
    operator to its own elements, sums the shared surface values with one
    exchange per operator application (and one for the diagonal), and forms
    inner products over its unique nodes with each shared node weighted by
    1 / (ranks holding it), reduced across ranks."""
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import paper_2501_13240_gb300 as sem
        N = case["N"]
        om = oracle.box_mesh(case["nel"], N, periodic=case["periodic"], dirichlet=case["dirichlet"],
                             deform_amp=0.1, kappa=np.full(9, 1.0), phi=np.array([0.3, 0.7, 1.1]))
        desc = sem.box_desc(case["nel"], N, periodic=case["periodic"], dirichlet=case["dirichlet"])
        n3 = (N + 1) ** 3
        e0, e1, _ = sem.sem_partition_info(desc, world, rank)
        gids, nshare = sem.sem_partition_interface(desc, world, rank)
        allg = np.unique(np.concatenate([sem.sem_partition_interface(desc, world, q)[0] for q in range(world)]))
        mine = slice(e0 * n3, e1 * n3)
        own = np.unique(om.l2g[mine])
        loc = np.searchsorted(own, om.l2g[mine])  # local node -> this rank's unique node
        at, slot = np.searchsorted(own, gids), np.searchsorted(allg, gids)
        wdot = np.ones(len(own))
        wdot[at] = 1.0 / nshare
        mk = om.mask[own].astype(np.float64)
        G = np.ascontiguousarray(om.G[:, mine])
        B = np.ascontiguousarray(om.B[mine])

        def exchange(part):
            buf = torch.zeros(len(allg), dtype=torch.float64)
            buf[slot] = torch.from_numpy(part[at])
            dist.all_reduce(buf)
            part[at] = buf.numpy()[slot]
            return part

        def assemble(vL):
            part = np.zeros(len(own))
            np.add.at(part, loc, vL)
            return exchange(part)

        def A(v):
            return mk * assemble(oracle.ax_local_raw(N, om.D, G, B, (mk * v)[loc], 1.0, h2))

        def dot(a, b):
            t = torch.tensor([float(np.sum(wdot * a * b))], dtype=torch.float64)
            dist.all_reduce(t)
            return float(t[0])

        dL = np.zeros(e1 * n3 - e0 * n3)
        oracle.lib().or_diag_local(e1 - e0, N, np.ascontiguousarray(om.D.ravel()), np.ascontiguousarray(G.ravel()),
                                   B, 1.0, float(h2), dL)
        d = assemble(dL)
        dinv = np.where(mk != 0, 1.0 / np.where(mk != 0, d, 1.0), 0.0)
        b_all = om.mask * np.random.default_rng(23).standard_normal(om.n_unique)
        ref = oracle.pcg(om, b_all, 1.0, h2, tol=1e-10, maxit=500)
        b = b_all[own]
        x = np.zeros_like(b)
        r = b.copy()
        bn = np.sqrt(dot(b, b))
        z = dinv * r
        p = z.copy()
        rho = dot(r, z)
        its = 0
        for its in range(1, 501):
            w = A(p)
            alpha = rho / dot(p, w)
            x += alpha * p
            r -= alpha * w
            if np.sqrt(dot(r, r)) <= 1e-10 * bn:
                break
            z = dinv * r
            rho1 = dot(r, z)
            p = z + (rho1 / rho) * p
            rho = rho1
        err = float(np.abs(x - ref.x[own]).max() / np.abs(ref.x).max())
        dd = float(np.abs(d - oracle.diag_assembled(om, 1.0, h2)[own]).max())
        queue.put((rank, its, ref.iterations, err, dd))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case,h2", [(0, 0.0), (1, 0.5), (2, 0.0)])
def test_partitioned_jacobi_pcg_matches_single_partition(world, case, h2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_pcg, args=(r, world, port, CASES[case], h2, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, its, ref_its, err, dd in sorted(res):
        assert abs(its - ref_its) <= 1, (rank, its, ref_its)
        assert err < 1e-9, (rank, err)
        assert dd < 1e-12, (rank, dd)
    assert len({r[1] for r in res}) == 1  # every rank stops at the same iteration


def _worker_peers(rank, world, port, case, queue):
    """Pairwise exchange over the neighbour plan: each rank trades its
    partial sums at the nodes it shares with each partner (point to point,
    no collective over all ranks) and adds them in ascending rank order, so
    both ranks of a pair hold the same bits."""
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import paper_2501_13240_gb300 as sem
        om = oracle.box_mesh(case["nel"], case["N"], periodic=case["periodic"], dirichlet=case["dirichlet"])
        desc = sem.box_desc(case["nel"], case["N"], periodic=case["periodic"], dirichlet=case["dirichlet"])
        n3 = (case["N"] + 1) ** 3
        e0, e1, ni = sem.sem_partition_info(desc, world, rank)
        gids, _ = sem.sem_partition_interface(desc, world, rank)
        mine = slice(e0 * n3, e1 * n3)
        own = np.unique(om.l2g[mine])
        peers = sem.sem_partition_peers(desc, world, rank)
        brute = []
        for q in range(world):
            a, b, _ = sem.sem_partition_info(desc, world, q)
            shared = np.intersect1d(own, om.l2g[a * n3:b * n3]) if q != rank else np.zeros(0)
            if len(shared):
                brute.append((q, shared))
        plan_ok = [p for p, _ in peers] == [q for q, _ in brute]
        nodes = {p: sem.sem_partition_peer_nodes(desc, world, rank, p) for p, _ in peers}
        plan_ok &= all(np.array_equal(nodes[q], s) and c == len(s) for (q, s), (_, c) in zip(brute, peers))
        plan_ok &= np.array_equal(np.unique(np.concatenate(list(nodes.values()) or [np.zeros(0, np.int64)])), gids)
        plan_ok &= sum(c for _, c in peers) == ni
        v = np.random.default_rng(29).standard_normal(om.n_local)
        part = np.zeros(om.n_unique)
        np.add.at(part, om.l2g[mine], v[mine])
        recv = {}
        reqs = []
        for p, _ in peers:
            recv[p] = torch.zeros(len(nodes[p]), dtype=torch.float64)
            reqs.append(dist.isend(torch.from_numpy(part[nodes[p]].copy()), p))
            reqs.append(dist.irecv(recv[p], p))
        for r in reqs:
            r.wait()
        total = part.copy()
        for p, _ in peers:
            mine_p, theirs = part[nodes[p]], recv[p].numpy()
            total[nodes[p]] = (mine_p + theirs) if rank < p else (theirs + mine_p)
        ref = oracle.qqt(om, v)[mine]
        err = float(np.abs(total[om.l2g[mine]] - ref).max() / np.abs(ref).max())
        # both ranks of each pair hold the same bits on the shared nodes
        back = {}
        reqs = []
        for p, _ in peers:
            back[p] = torch.zeros(len(nodes[p]), dtype=torch.float64)
            reqs.append(dist.isend(torch.from_numpy(total[nodes[p]].copy()), p))
            reqs.append(dist.irecv(back[p], p))
        for r in reqs:
            r.wait()
        same = all(np.array_equal(back[p].numpy(), total[nodes[p]]) for p, _ in peers)
        queue.put((rank, bool(plan_ok), err, bool(same), len(peers)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_pairwise_exchange_over_the_neighbour_plan(world, case):
    if world > CASES[case]["nel"][2]:
        pytest.skip("more ranks than element planes")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_peers, args=(r, world, port, CASES[case], q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    periodic_z = CASES[case]["periodic"][2]
    for rank, plan_ok, err, same, npeers in sorted(res):
        assert plan_ok, rank
        assert err < 1e-14, (rank, err)
        assert same, rank
        interior = 0 < rank < world - 1
        assert npeers == (1 if world == 2 else 2 if (interior or periodic_z) else 1), (rank, npeers)


def test_neighbour_plan_arguments():
    import paper_2501_13240_gb300 as sem
    d = sem.box_desc((2, 2, 4), 3, periodic=(0, 0, 1), dirichlet=(1, 1, 1, 1, 0, 0))
    assert sem.sem_partition_peers(d, 1, 0) == []  # one rank: the periodic wrap is its own
    assert sem.sem_partition_peers(d, 2, 0) == [(1, 2 * 7 * 7)]  # the middle plane and the wrapped one
    with pytest.raises(sem.SemError):
        sem.sem_partition_peer_nodes(d, 2, 0, 0)
    with pytest.raises(sem.SemError):
        sem.sem_partition_peer_nodes(d, 2, 0, 2)
    assert len(sem.sem_partition_peer_nodes(d, 4, 0, 2)) == 0  # not a partner: nothing shared


def _worker_overlap(rank, world, port, case, queue):
    """The overlapped schedule of Sec. 2.2 over the surface-element plan:
    surface elements first, then the pairwise exchange of the interface
    partial sums started (non-blocking) while the interior elements are
    summed, then the received partial sums added."""
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import paper_2501_13240_gb300 as sem
        om = oracle.box_mesh(case["nel"], case["N"], periodic=case["periodic"], dirichlet=case["dirichlet"])
        desc = sem.box_desc(case["nel"], case["N"], periodic=case["periodic"], dirichlet=case["dirichlet"])
        n3 = (case["N"] + 1) ** 3
        e0, e1, _ = sem.sem_partition_info(desc, world, rank)
        gids, _ = sem.sem_partition_interface(desc, world, rank)
        surf = sem.sem_partition_surface(desc, world, rank)
        l2g = om.l2g.reshape(om.E, n3)
        brute = np.array([e for e in range(e0, e1) if np.intersect1d(l2g[e], gids).size], dtype=np.int64)
        plan_ok = np.array_equal(surf, brute)
        inner = np.setdiff1d(np.arange(e0, e1), surf)
        v = np.random.default_rng(31).standard_normal(om.n_local).reshape(om.E, n3)
        part = np.zeros(om.n_unique)
        np.add.at(part, l2g[surf].ravel(), v[surf].ravel())  # surface pass
        full = np.zeros(om.n_unique)
        np.add.at(full, l2g[e0:e1].ravel(), v[e0:e1].ravel())
        plan_ok &= np.array_equal(part[gids], full[gids])  # interface sums complete after the surface pass
        peers = [p for p, _ in sem.sem_partition_peers(desc, world, rank)]
        nodes = {p: sem.sem_partition_peer_nodes(desc, world, rank, p) for p in peers}
        recv = {p: torch.zeros(len(nodes[p]), dtype=torch.float64) for p in peers}
        reqs = []
        for p in peers:
            reqs.append(dist.isend(torch.from_numpy(part[nodes[p]].copy()), p))
            reqs.append(dist.irecv(recv[p], p))
        np.add.at(part, l2g[inner].ravel(), v[inner].ravel())  # interior pass while the exchange is in flight
        for r in reqs:
            r.wait()
        for p in peers:
            mine_p, theirs = part[nodes[p]], recv[p].numpy()
            part[nodes[p]] = (mine_p + theirs) if rank < p else (theirs + mine_p)
        ref = oracle.qqt(om, v.ravel())[e0 * n3:e1 * n3]
        err = float(np.abs(part[l2g[e0:e1].ravel()] - ref).max() / np.abs(ref).max())
        queue.put((rank, bool(plan_ok), err, len(surf) // (case["nel"][0] * case["nel"][1]), e1 - e0))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_overlapped_exchange_over_the_surface_plan(world, case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_overlap, args=(r, world, port, CASES[case], q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    periodic_z = CASES[case]["periodic"][2]
    plane = CASES[case]["nel"][0] * CASES[case]["nel"][1]
    for rank, plan_ok, err, nplanes, nelem in sorted(res):
        assert plan_ok, rank
        assert err < 1e-14, (rank, err)
        shared_sides = int(rank > 0 or bool(periodic_z)) + int(rank < world - 1 or bool(periodic_z))
        assert nplanes == min(shared_sides, nelem // plane), (rank, nplanes)


def test_surface_plan_single_rank_and_arguments():
    import paper_2501_13240_gb300 as sem
    d = sem.box_desc((2, 3, 4), 3, periodic=(0, 0, 1), dirichlet=(1, 1, 1, 1, 0, 0))
    assert len(sem.sem_partition_surface(d, 1, 0)) == 0  # one rank: no interface, all elements interior
    assert np.array_equal(sem.sem_partition_surface(d, 4, 1), np.arange(6, 12))  # one plane, both sides
    assert np.array_equal(sem.sem_partition_surface(d, 2, 0), np.arange(0, 12))  # periodic: planes 0 and 1
    with pytest.raises(sem.SemError):
        sem.sem_partition_surface(d, 5, 0)
