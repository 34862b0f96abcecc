"""Property tests of the element-slab partition plan (host C code, Sec. 2.2:
one rank per GPU, shared surface values summed across ranks) on random box
sizes, orders, periodicity and rank counts, against brute force from the
oracle's node numbering: the ranks' element ranges tile the mesh, and each
rank's interface nodes, holder counts, exchange partners, shared-node lists
and surface elements are exactly the ones the node sets imply. CPU only."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
import paper_2501_13240_gb300 as sem  # noqa: E402


@st.composite
def plans(draw):
    nel = (draw(st.integers(1, 3)), draw(st.integers(1, 3)), draw(st.integers(1, 6)))
    N = draw(st.integers(1, 4))
    periodic = tuple(draw(st.integers(0, 1)) for _ in range(3))
    nranks = draw(st.integers(1, nel[2]))
    return nel, N, periodic, nranks


@settings(max_examples=200, deadline=None)
@given(plans())
def test_partition_plan_equals_brute_force(plan):
    nel, N, periodic, P = plan
    om = oracle.box_mesh(nel, N, periodic=periodic, dirichlet=(0,) * 6, geometry=False)
    d = sem.box_desc(nel, N, periodic=periodic, dirichlet=(0,) * 6)
    n3 = (N + 1) ** 3
    E = nel[0] * nel[1] * nel[2]
    l2g = om.l2g.reshape(E, n3)
    ranges = [sem.sem_partition_info(d, P, r)[:2] for r in range(P)]
    assert ranges[0][0] == 0 and ranges[-1][1] == E
    assert all(ranges[r][1] == ranges[r + 1][0] and ranges[r][0] < ranges[r][1] for r in range(P - 1))
    nodes = [np.unique(l2g[a:b]) for a, b in ranges]
    holders = np.zeros(om.n_unique, dtype=np.int64)
    for ns in nodes:
        holders[ns] += 1
    assert holders.max() <= 2  # slabs: a node is held by at most two ranks
    for r, (a, b) in enumerate(ranges):
        gids, nshare = sem.sem_partition_interface(d, P, r)
        iface = nodes[r][holders[nodes[r]] > 1]
        assert np.array_equal(gids, iface)
        assert np.array_equal(nshare, holders[gids])
        assert sem.sem_partition_info(d, P, r)[2] == len(iface)
        peers = sem.sem_partition_peers(d, P, r)
        brute = [(q, np.intersect1d(nodes[r], nodes[q])) for q in range(P) if q != r]
        brute = [(q, s) for q, s in brute if len(s)]
        assert [p for p, _ in peers] == [q for q, _ in brute]
        for (q, s), (_, c) in zip(brute, peers):
            assert c == len(s)
            assert np.array_equal(sem.sem_partition_peer_nodes(d, P, r, q), s)
        surf = sem.sem_partition_surface(d, P, r)
        assert np.array_equal(surf, [e for e in range(a, b) if np.intersect1d(l2g[e], iface).size])
