"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs (Sec. 2.2: GLL set-up, chain-rule geometry,
matrix-free Ax, direct stiffness summation, Jacobi-PCG).

Tolerances: index maps bit-exact; floating point 1e-12 relative in the max
norm (max |gpu - oracle| <= 1e-12 max |oracle|), the FP64 parity bar."""
import numpy as np
import pytest

import oracle
import workloads
from workloads import POISSON_4, AX_GS_64, BoxWorkload

torch = pytest.importorskip("torch")
import paper_2501_13240_gb300 as sem  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL = 1e-12
KAPPA = np.array([[1.0, 2.0, 1.0], [2.0, 1.0, 1.0], [1.0, 1.0, 2.0]])
PHI = np.array([0.3, 1.7, 4.1])


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


# meshes small enough for the oracle, spanning several CTAs with ragged tails
MESHES = [
    dict(nel=(5, 3, 3), N=7, deform=0.05),                        # 45 elements: ragged last CTA
    dict(nel=(4, 4, 4), N=7, deform=0.0),                         # the poisson_4 mesh
    dict(nel=(3, 2, 2), N=4, deform=0.05, L=(1.0, 2.0, 0.5)),
    dict(nel=(2, 3, 4), N=9, deform=0.04, periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), stretch=2.0),
    dict(nel=(1, 1, 1), N=1, deform=0.0),
    dict(nel=(9, 7, 5), N=1, deform=0.05, periodic=(1, 0, 0), dirichlet=(0, 0, 1, 1, 1, 1)),  # element matrices
    dict(nel=(2, 2, 2), N=10, deform=0.05),
    dict(nel=(3, 3, 2), N=2, deform=0.05, periodic=(1, 0, 1), dirichlet=(0, 0, 1, 1, 0, 0)),
    # even point counts NP = 4, 6: the packed double-float operator with two and
    # eight elements per CTA (idle padding threads at NP = 6)
    dict(nel=(3, 4, 3), N=3, deform=0.06, periodic=(0, 1, 0), dirichlet=(1, 1, 0, 0, 1, 1)),
    dict(nel=(4, 2, 3), N=5, deform=0.05, L=(2.0, 1.0, 1.5)),
]


def make(spec):
    kw = dict(nel=spec["nel"], N=spec["N"], L=spec.get("L", (1.0, 1.0, 1.0)), periodic=spec.get("periodic", (0, 0, 0)),
              dirichlet=spec.get("dirichlet", (1,) * 6), z_stretch=spec.get("stretch", 0.0),
              deform_amp=spec["deform"], kappa=KAPPA, phi=PHI)
    om = oracle.box_mesh(kw["nel"], kw["N"], kw["L"], kw["periodic"], kw["dirichlet"], kw["z_stretch"],
                         kw["deform_amp"], KAPPA, PHI)
    gm = sem.sem_mesh_create_box(**kw)
    return om, gm


@pytest.fixture(scope="module", params=range(len(MESHES)), ids=lambda i: "mesh%d" % i)
def pair(request):
    om, gm = make(MESHES[request.param])
    yield om, gm
    gm.destroy()


def test_maps_bit_exact(pair):
    om, gm = pair
    assert gm.n_local == om.n_local and gm.n_unique == om.n_unique and gm.E == om.E
    l2g, mask = gm.maps()
    np.testing.assert_array_equal(l2g.astype(np.int64), om.l2g)
    np.testing.assert_array_equal(mask, om.mask)
    off, perm = gm.gs_tables()
    assert off[0] == 0 and off[-1] == om.n_local
    assert np.all(np.diff(off) >= 1)
    np.testing.assert_array_equal(np.sort(perm), np.arange(om.n_local))
    seg = np.repeat(np.arange(om.n_unique), np.diff(off))
    np.testing.assert_array_equal(om.l2g[perm], seg)
    same = seg[1:] == seg[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])  # ascending within a segment
    np.testing.assert_array_equal(host(gm.field("mult")), om.mult)


def test_geometry(pair):
    om, gm = pair
    n3 = (om.N + 1) ** 3
    for name, ref in (("X", om.X), ("Y", om.Y), ("Z", om.Z), ("B", om.B)):
        assert rel_err(host(gm.field(name)), ref) < RTOL, name
    G = host(gm.field("G")).reshape(om.E, 6, n3).transpose(1, 0, 2).reshape(6, -1)
    assert rel_err(G, om.G) < 1e-11
    assert abs(gm.detJ_min - om.detJ_min) <= 1e-12 * abs(om.detJ_min)


PRECS = [sem.SEM_PREC_FP64, sem.SEM_PREC_DF64]
PREC_IDS = ["fp64", "df64"]


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.37, 12.5), (0.0, 2.0)])
def test_ax_local(pair, h1, h2, prec):
    om, gm = pair
    u = np.random.default_rng(11).uniform(-1, 1, om.n_local)
    w = torch.empty(om.n_local, dtype=torch.float64, device="cuda")
    sem.sem_ax_apply(gm, h1, h2, dev(u), w, precision=prec)
    assert rel_err(host(w), oracle.ax_local(om, u, h1, h2)) < RTOL


@pytest.mark.parametrize("apply_mask", [False, True])
def test_gs_op(pair, apply_mask):
    om, gm = pair
    v = np.random.default_rng(12).standard_normal(om.n_local)
    t = dev(v)
    sem.sem_gs_op(gm, t, apply_mask)
    assert rel_err(host(t), oracle.qqt(om, v, apply_mask)) < 1e-15


def test_gather_scatter(pair):
    om, gm = pair
    v = np.random.default_rng(13).standard_normal(om.n_local)
    g = torch.empty(om.n_unique, dtype=torch.float64, device="cuda")
    sem.sem_gather(gm, dev(v), g)
    assert rel_err(host(g), oracle.gather_sum(om, v)) < 1e-15
    ug = np.random.default_rng(14).standard_normal(om.n_unique)
    L = torch.empty(om.n_local, dtype=torch.float64, device="cuda")
    sem.sem_scatter(gm, dev(ug), L)
    np.testing.assert_array_equal(host(L), oracle.scatter(om, ug))


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.37, 12.5)])
def test_ax_assembled(pair, h1, h2, prec):
    om, gm = pair
    ug = np.random.default_rng(15).uniform(-1, 1, om.n_unique)
    w = torch.empty(om.n_unique, dtype=torch.float64, device="cuda")
    sem.sem_ax_assembled(gm, h1, h2, dev(ug), w, precision=prec)
    assert rel_err(host(w), oracle.apply_assembled(om, ug, h1, h2)) < RTOL


@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.37, 12.5)])
def test_jacobi_inv(pair, h1, h2):
    om, gm = pair
    d = torch.empty(om.n_unique, dtype=torch.float64, device="cuda")
    sem.sem_jacobi_inv(gm, h1, h2, d)
    assert rel_err(host(d), oracle.jacobi_inv(om, h1, h2)) < RTOL


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.5, 40.0)])
def test_pcg_solve(pair, h1, h2, prec):
    om, gm = pair
    if om.mask.sum() == 0:
        pytest.skip("no free nodes")
    b = np.random.default_rng(16).standard_normal(om.n_unique) * om.mask
    ref = oracle.pcg(om, b, h1, h2, tol=1e-10, maxit=3000)
    x = torch.zeros(om.n_unique, dtype=torch.float64, device="cuda")
    st = sem.sem_pcg_solve(gm, h1, h2, dev(b), x, tol=1e-10, maxit=3000, precision=prec)
    assert st["status"] == 0 and ref.converged
    assert abs(st["iterations"] - ref.iterations) <= 1, (st, ref.iterations)
    assert st["rel_residual"] <= 1e-10
    assert rel_err(host(x), ref.x) < 1e-9


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_pcg_from_initial_guess(pair, prec):
    """r_0 = b - A x0, the stopping test still ||r|| <= tol ||b||: iterations
    and solution as the oracle's from the same guess; a guess that already
    meets the tolerance returns it unchanged after 0 iterations; values on
    Dirichlet nodes are kept (the operator ignores them); b = 0 gives x = 0."""
    om, gm = pair
    if om.mask.sum() == 0:
        pytest.skip("no free nodes")
    h1, h2 = 0.5, 40.0
    rng = np.random.default_rng(17)
    b = rng.standard_normal(om.n_unique) * om.mask
    tight = oracle.pcg(om, b, h1, h2, tol=1e-12, maxit=3000)
    x0 = tight.x + 1e-3 * rng.standard_normal(om.n_unique) * np.abs(tight.x).max()
    ref = oracle.pcg(om, b, h1, h2, tol=1e-10, maxit=3000, x0=x0)
    x = dev(x0)
    st = sem.sem_pcg_solve(gm, h1, h2, dev(b), x, tol=1e-10, maxit=3000, precision=prec, initial_guess=True)
    assert st["status"] == 0 and ref.converged and ref.iterations > 0
    assert abs(st["iterations"] - ref.iterations) <= 1, (st, ref.iterations)
    assert rel_err(host(x), ref.x) < 1e-9
    # the oracle's guess meets a looser tolerance: nothing to do
    loose = oracle.pcg(om, b, h1, h2, tol=1e-8, maxit=3000, x0=tight.x)
    assert loose.iterations == 0
    x = dev(tight.x)
    st = sem.sem_pcg_solve(gm, h1, h2, dev(b), x, tol=1e-8, maxit=3000, precision=prec, initial_guess=True)
    assert st["status"] == 0 and st["iterations"] == 0 and st["rel_residual"] <= 1e-8
    np.testing.assert_array_equal(host(x), tight.x)
    # b = 0: x = 0 whatever the guess
    x = dev(x0)
    st = sem.sem_pcg_solve(gm, h1, h2, dev(0.0 * b), x, precision=prec, initial_guess=True)
    assert st["iterations"] == 0 and st["status"] == 0 and float(x.abs().max()) == 0.0


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_pcg_guess_edge_cases(prec):
    """A non-finite guess ends in SEM_ERR_BREAKDOWN with 0 iterations (not a
    silent result); the flag must be 0 or 1; a zero guess is the cold start
    (same iterations and solution as initial_guess = False)."""
    gm = sem.sem_mesh_create_box((2, 2, 2), 5, deform_amp=0.05)
    om = oracle.box_mesh((2, 2, 2), 5, deform_amp=0.05)
    b = np.random.default_rng(19).standard_normal(om.n_unique) * om.mask
    x = torch.zeros(om.n_unique, dtype=torch.float64, device="cuda")
    x[om.n_unique // 2] = float("nan")
    st = sem.sem_pcg_solve(gm, 1.0, 0.0, dev(b), x, precision=prec, initial_guess=True, raise_on_error=False)
    assert st["status"] == sem.SEM_ERR_BREAKDOWN and st["iterations"] == 0
    cold = torch.zeros_like(x)
    st0 = sem.sem_pcg_solve(gm, 1.0, 0.0, dev(b), cold, tol=1e-10, precision=prec)
    warm = torch.zeros_like(x)
    st1 = sem.sem_pcg_solve(gm, 1.0, 0.0, dev(b), warm, tol=1e-10, precision=prec, initial_guess=True)
    assert st1["iterations"] == st0["iterations"]
    assert rel_err(host(warm), host(cold)) < 1e-12
    gm.destroy()


def test_pcg_initial_guess_pure_neumann():
    """The singular operator (mask_mode 1, right-hand side of zero mean) from
    a guess, as the pressure solve runs it, against the oracle's iteration."""
    nel, N = (3, 2, 2), 5
    kw = dict(periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), deform_amp=0.05)
    om = oracle.box_mesh(nel, N, **kw)
    gm = sem.sem_mesh_create_box(nel, N, **kw)
    free = oracle.Mesh(om.nel, om.N, om.periodic, om.dirichlet, om.xi, om.rho, om.D, om.X, om.Y, om.Z, om.G, om.B,
                       om.l2g, np.ones(om.n_unique, dtype=np.uint8), om.n_unique, om.detJ_min, om.L)
    rng = np.random.default_rng(18)
    b = rng.standard_normal(om.n_unique)
    b -= b.mean()
    apply = lambda v: oracle.gather_sum(free, oracle.ax_local(free, oracle.scatter(free, v), 1.0, 0.0))  # noqa: E731
    x0 = rng.standard_normal(om.n_unique)
    ref = oracle.pcg(free, b, 1.0, 0.0, tol=1e-10, maxit=3000, apply=apply, x0=x0)
    for prec in PRECS:
        x = dev(x0)
        st = sem.sem_pcg_solve(gm, 1.0, 0.0, dev(b), x, tol=1e-10, maxit=3000, precision=prec, mask_mode=1,
                               initial_guess=True)
        assert st["status"] == 0 and abs(st["iterations"] - ref.iterations) <= 1, (st, ref.iterations)
        xg = host(x)  # x is fixed up to a constant: compare the zero-mean parts
        assert rel_err(xg - xg.mean(), ref.x - ref.x.mean()) < 1e-9
    gm.destroy()


def test_poisson_4_manufactured_solution():
    """The poisson_4 workload: Jacobi-PCG to 1e-10 reaches the oracle's solution
    and iteration count, and the spectral-element error of u = sin sin sin."""
    om = oracle.mesh_from_workload(POISSON_4)
    gm = sem.mesh_from_workload(POISSON_4)
    b = oracle.poisson_rhs(om)
    ref = oracle.pcg(om, b, tol=1e-10, maxit=1000)
    x = torch.zeros(om.n_unique, dtype=torch.float64, device="cuda")
    st = sem.sem_pcg_solve(gm, 1.0, 0.0, dev(b), x, tol=1e-10, maxit=1000)
    assert st["status"] == 0
    assert abs(st["iterations"] - ref.iterations) <= 1
    xg = host(x)
    assert rel_err(xg, ref.x) < 1e-10
    err = np.abs(oracle.scatter(om, xg) - oracle.manufactured_u(om)).max()
    assert err < 1e-5
    gm.destroy()


def test_large_grid_stride_assembled():
    """More elements than the fixed assembled grid holds (each CTA loops)."""
    spec = dict(nel=(24, 24, 20), N=7, deform=0.1)
    om, gm = make(spec)
    ug = np.random.default_rng(21).uniform(-1, 1, om.n_unique)
    ref = oracle.apply_assembled(om, ug)
    for prec in PRECS:
        w = torch.empty(om.n_unique, dtype=torch.float64, device="cuda")
        sem.sem_ax_assembled(gm, 1.0, 0.0, dev(ug), w, precision=prec)
        assert rel_err(host(w), ref) < RTOL, prec
    gm.destroy()


WIDE = [1.0, 1e-20, 3.7e25, 2.0 ** -60, 1e40, 1e-35, 1e200, 1e-200]


@pytest.mark.parametrize("scale", WIDE)
@pytest.mark.parametrize("N", [7, 4, 1])
def test_df64_wide_magnitudes(scale, N):
    """The double-float operators (local and assembled, Helmholtz and
    Poisson) keep binary64-level accuracy for inputs far outside the binary32
    exponent range: each element is computed at the power-of-two scale of its
    largest input. Nothing comes back infinite or flushed to zero."""
    spec = dict(nel=(3, 2, 2), N=N, deform=0.05)
    om, gm = make(spec)
    rng = np.random.default_rng(22)
    u = rng.uniform(-1, 1, om.n_local) * scale
    w = torch.empty(om.n_local, dtype=torch.float64, device="cuda")
    sem.sem_ax_apply(gm, 1.0, 0.0, dev(u), w, precision=sem.SEM_PREC_DF64)
    ref = oracle.ax_local(om, u)
    assert np.isfinite(host(w)).all() and rel_err(host(w), ref) < RTOL
    ug = rng.uniform(-1, 1, om.n_unique) * scale
    for h1, h2 in [(1.0, 0.0), (0.7, 30.0)]:
        wg = torch.empty(om.n_unique, dtype=torch.float64, device="cuda")
        sem.sem_ax_assembled(gm, h1, h2, dev(ug), wg, precision=sem.SEM_PREC_DF64)
        refg = oracle.apply_assembled(om, ug, h1, h2)
        got = host(wg)
        assert np.isfinite(got).all() and rel_err(got, refg) < RTOL, (h1, h2)
        assert (got[refg != 0] != 0).all()
    gm.destroy()


# ------------------------------------------------------------------ edge cases
def test_invalid_arguments_are_rejected():
    bad = [dict(nel=(0, 1, 1), N=3), dict(nel=(1, 1, 1), N=0), dict(nel=(1, 1, 1), N=11),
           dict(nel=(1, 2, 2), N=3, periodic=(1, 0, 0)), dict(nel=(1, 1, 1), N=3, L=(1.0, -1.0, 1.0))]
    for kw in bad:
        with pytest.raises(sem.SemError) as ei:
            sem.sem_mesh_create_box(**kw)
        assert ei.value.code == sem.SEM_ERR_INVALID_ARG, kw
    # an inverted mesh (deformation too large) is rejected, not silently used
    with pytest.raises(sem.SemError) as ei:
        sem.sem_mesh_create_box((1, 1, 1), 5, deform_amp=0.5, kappa=KAPPA, phi=PHI)
    assert ei.value.code == sem.SEM_ERR_INVALID_ARG and "Jacobian" in str(ei.value)
    gm = sem.sem_mesh_create_box((2, 2, 2), 3)
    u = torch.zeros(gm.n_local, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError):
        sem.sem_ax_apply(gm, 1.0, 0.0, u, u)  # aliasing rejected
    with pytest.raises(sem.SemError):
        sem.sem_ax_apply(gm, 1.0, 0.0, u, torch.zeros_like(u), precision=7)
    b = torch.zeros(gm.n_unique, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError):
        sem.sem_pcg_solve(gm, 0.0, 0.0, b, torch.zeros_like(b))
    gm.destroy()


def test_pcg_zero_rhs_and_maxit():
    gm = sem.sem_mesh_create_box((2, 2, 2), 4)
    b = torch.zeros(gm.n_unique, dtype=torch.float64, device="cuda")
    x = torch.full_like(b, 5.0)
    st = sem.sem_pcg_solve(gm, 1.0, 0.0, b, x)
    assert st["iterations"] == 0 and st["status"] == 0 and float(x.abs().max()) == 0.0
    om = oracle.box_mesh((2, 2, 2), 4)
    bb = np.random.default_rng(3).standard_normal(om.n_unique) * om.mask
    st = sem.sem_pcg_solve(gm, 1.0, 0.0, dev(bb), x, tol=1e-14, maxit=3, raise_on_error=False)
    assert st["status"] == sem.SEM_ERR_NOT_CONVERGED and st["iterations"] == 3
    ref = oracle.pcg(om, bb, tol=1e-14, maxit=3)
    assert rel_err(host(x), ref.x) < 1e-10
    gm.destroy()


def test_nan_input_reports_breakdown():
    """Fault injection on the host: a NaN in the right-hand side ends the
    solve with SEM_ERR_BREAKDOWN instead of iterating on garbage."""
    gm = sem.sem_mesh_create_box((2, 2, 2), 3)
    b = torch.zeros(gm.n_unique, dtype=torch.float64, device="cuda")
    b[gm.n_unique // 2] = float("nan")
    st = sem.sem_pcg_solve(gm, 1.0, 0.0, b, torch.zeros_like(b), raise_on_error=False)
    assert st["status"] == sem.SEM_ERR_BREAKDOWN
    gm.destroy()


# ------------------------------------------------------------------ full size
def test_ax_gs_64_full_size_spot_check():
    """The 64^3-element, N = 7 deformed mesh of the throughput benchmark, in the
    launch configuration the benchmark times: sampled elements of the local
    operator and sampled unique nodes of the assembled operator against the
    oracle computed element by element."""
    w = AX_GS_64
    gm = sem.mesh_from_workload(w)
    assert gm.n_local == w.n_local and gm.n_unique == w.n_unique
    ug = workloads.unique_field(w.n_unique)
    ug_d = dev(ug)
    uL = torch.empty(gm.n_local, dtype=torch.float64, device="cuda")
    sem.sem_scatter(gm, ug_d, uL)
    wL = torch.empty_like(uL)
    sem.sem_ax_apply(gm, 1.0, 0.0, uL, wL)
    wg = torch.empty_like(ug_d)
    sem.sem_ax_assembled(gm, 1.0, 0.0, ug_d, wg)
    wL2 = torch.empty_like(uL)
    sem.sem_ax_apply(gm, 1.0, 0.0, uL, wL2, precision=sem.SEM_PREC_DF64)
    wg2 = torch.empty_like(ug_d)
    sem.sem_ax_assembled(gm, 1.0, 0.0, ug_d, wg2, precision=sem.SEM_PREC_DF64)
    l2g, mask = gm.maps()
    n3 = 512
    rng = np.random.default_rng(5)
    elems = np.unique(np.concatenate([[0, w.E - 1], rng.integers(0, w.E, 60)]))
    X, Y, Z, G, B, D = oracle.element_subset(w, elems)
    idx = (elems[:, None] * n3 + np.arange(n3)[None, :]).ravel()
    u_sub = ug[l2g[idx]]
    ref = oracle.ax_local_raw(w.N, D, G, B, u_sub)
    got = host(wL)[idx]
    assert rel_err(got, ref) < RTOL
    assert rel_err(host(wL2)[idx], ref) < RTOL
    # geometry of the sampled elements
    Gg = host(gm.field("G")).reshape(w.E, 6, n3)[elems].transpose(1, 0, 2).reshape(6, -1)
    assert rel_err(Gg, G) < 1e-11
    # assembled values at sampled unique nodes: sum over every element that
    # holds a copy of the node (found from the l2g map)
    gsel = l2g[idx[rng.integers(0, len(idx), 40)]]
    gsel = gsel[mask[gsel] == 1]
    holders = np.unique(np.nonzero(np.isin(l2g, gsel))[0] // n3)
    X2, Y2, Z2, G2, B2, _ = oracle.element_subset(w, holders)
    idx2 = (holders[:, None] * n3 + np.arange(n3)[None, :]).ravel()
    w2 = oracle.ax_local_raw(w.N, D, G2, B2, ug[l2g[idx2]] * mask[l2g[idx2]])
    acc = np.zeros(w.n_unique)
    np.add.at(acc, l2g[idx2], w2)
    assert rel_err(host(wg)[gsel], acc[gsel]) < RTOL
    assert rel_err(host(wg2)[gsel], acc[gsel]) < RTOL
    # and the two precisions agree everywhere (norm-wise)
    assert rel_err(host(wg2), host(wg)) < RTOL
    gm.destroy()
