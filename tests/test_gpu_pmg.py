"""GPU parity of the p-multigrid preconditioner and the mixed-precision
flexible CG (Sec. 2.2: p-multigrid, 4th-kind Chebyshev smoothing, FP32
preconditioner) against the binary64 oracle. Smoothing levels run in binary32
(or bfloat16 geometry), so component parity is checked at binary32 level and
the solve against binary64 residuals and solutions."""
import numpy as np
import pytest

import oracle
from oracle import pmg
import workloads

torch = pytest.importorskip("torch")
import paper_2501_13240_gb300 as sem  # noqa: E402

pytestmark = pytest.mark.gpu

KAPPA = np.array([[1.0, 2.0, 1.0], [2.0, 1.0, 1.0], [1.0, 1.0, 2.0]])
PHI = np.array([0.3, 1.7, 4.1])


def rel_err(a, b):
    s = np.abs(b).max()
    return np.abs(np.asarray(a) - b).max() / (s if s > 0 else 1.0)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


CASES = [(((4, 3, 3), 0.05), (7, 3, 1)), (((3, 3, 2), 0.0), (7, 3, 1)), (((2, 3, 2), 0.05), (6, 3, 1))]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=lambda i: "case%d" % i)
def hier(request):
    (nel, deform), orders = CASES[request.param]
    box = dict(nel=nel, deform_amp=deform, kappa=KAPPA, phi=PHI)
    pm = pmg.PMG(box, orders=orders)
    gm = sem.sem_mesh_create_box(nel, orders[0], deform_amp=deform, kappa=KAPPA, phi=PHI)
    gp = sem.sem_pmg_create(gm, orders=orders)
    yield pm, gm, gp
    gp.destroy()
    gm.destroy()


def test_lambda_estimates(hier):
    pm, gm, gp = hier
    for l in range(len(pm.levels) - 1):
        assert abs(gp.lam(l) - pm.levels[l].lam) <= 1e-4 * pm.levels[l].lam


def test_transfer_operators(hier):
    pm, gm, gp = hier
    rng = np.random.default_rng(4)
    for l in range(len(pm.levels) - 1):
        mf, mc = pm.levels[l].m, pm.levels[l + 1].m
        uc = rng.standard_normal(mc.n_unique) * mc.mask
        uf = torch.empty(mf.n_unique, dtype=torch.float64, device="cuda")
        sem.sem_pmg_prolong(gp, l, dev(uc), uf)
        assert rel_err(host(uf), pm.prolong(l, uc)) < 2e-6
        rf = rng.standard_normal(mf.n_unique) * mf.mask
        rc = torch.empty(mc.n_unique, dtype=torch.float64, device="cuda")
        sem.sem_pmg_restrict(gp, l, dev(rf), rc)
        assert rel_err(host(rc), pm.restrict(l, rf) * mc.mask) < 2e-6


def test_vcycle(hier):
    pm, gm, gp = hier
    m = pm.levels[0].m
    r = np.random.default_rng(6).standard_normal(m.n_unique) * m.mask
    z = torch.empty(m.n_unique, dtype=torch.float64, device="cuda")
    sem.sem_pmg_vcycle(gp, dev(r), z)
    # binary32 smoothing against the binary64 oracle: each operator output
    # is a sum of about 100 binary32 terms (worst case 100 x 2^-24 = 6e-6 of
    # |A||v|); measured about 1e-7 of max|z| on these meshes
    assert rel_err(host(z), pm.vcycle(r)) < 1e-5


@pytest.mark.parametrize("prec", [sem.SEM_PREC_DF64, sem.SEM_PREC_FP64], ids=["df64", "fp64"])
def test_mixed_solve_reaches_binary64_tolerance(hier, prec):
    pm, gm, gp = hier
    m = pm.levels[0].m
    b = oracle.poisson_rhs(m) if m.detJ_min > 0 else None
    x = torch.zeros(m.n_unique, dtype=torch.float64, device="cuda")
    st = sem.sem_pmg_pcg_solve(gp, dev(b), x, tol=1e-8, maxit=200, precision=prec)
    assert st["status"] == 0
    xg = host(x)
    true_res = np.linalg.norm(b - oracle.apply_assembled(m, xg)) / np.linalg.norm(b)
    assert true_res < 1.05e-8, true_res
    ref = pmg.fcg(pm, b, tol=1e-8)
    assert abs(st["iterations"] - ref.iterations) <= 2, (st, ref.iterations)
    tight = oracle.pcg(m, b, tol=1e-13, maxit=5000)
    assert rel_err(xg, tight.x) < 1e-6


@pytest.mark.parametrize("prec", [sem.SEM_PREC_DF64, sem.SEM_PREC_FP64], ids=["df64", "fp64"])
def test_fcg_from_initial_guess(hier, prec):
    """The flexible CG from a guess near the solution reaches the binary64
    tolerance in fewer iterations than from zero; a guess that already meets
    the tolerance is returned unchanged after 0 iterations."""
    pm, gm, gp = hier
    m = pm.levels[0].m
    b = oracle.poisson_rhs(m)
    tight = oracle.pcg(m, b, tol=1e-13, maxit=5000)
    x = torch.zeros(m.n_unique, dtype=torch.float64, device="cuda")
    cold = sem.sem_pmg_pcg_solve(gp, dev(b), x, tol=1e-10, maxit=200, precision=prec)
    x0 = tight.x * (1.0 + 1e-4 * np.random.default_rng(8).standard_normal(m.n_unique))
    x = dev(x0)
    st = sem.sem_pmg_pcg_solve(gp, dev(b), x, tol=1e-10, maxit=200, precision=prec, initial_guess=True)
    assert st["status"] == 0 and 0 < st["iterations"] < cold["iterations"], (st, cold)
    xg = host(x)
    assert np.linalg.norm(b - oracle.apply_assembled(m, xg)) / np.linalg.norm(b) < 1.05e-10
    assert rel_err(xg, tight.x) < 1e-8
    x = dev(tight.x)
    st = sem.sem_pmg_pcg_solve(gp, dev(b), x, tol=1e-8, maxit=200, precision=prec, initial_guess=True)
    assert st["status"] == 0 and st["iterations"] == 0
    np.testing.assert_array_equal(host(x), tight.x)


def bf16_round(x):
    """binary64 values rounded to the nearest bfloat16 (8 significant bits,
    ties to even), computed exactly on the bits: the rounding of the
    operator's inputs, applied before the oracle sees them"""
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)
    lsb = (b >> np.uint64(45)) & np.uint64(1)
    return ((b + np.uint64((1 << 44) - 1) + lsb) & ~np.uint64((1 << 45) - 1)).view(np.float64)


def test_bf16_round_helper():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -(1.0 + 2.0 ** -9), 3.0 + 2.0 ** -7 + 2.0 ** -30])
    np.testing.assert_array_equal(bf16_round(x), [1.0, 1.0, 1.0 + 2.0 ** -7, -1.0, 3.0 + 2.0 ** -6])


@pytest.mark.parametrize("h2", [0.0, 3.0], ids=["poisson", "helmholtz"])
@pytest.mark.parametrize("nel", [(3, 3, 2), (4, 3, 3)], ids=["18el", "36el"])
def test_bf16_tensor_core_level_operator(nel, h2):
    """The N = 7 bfloat16 smoothing operator (tensor cores, two-part bfloat16
    operands, binary32 accumulation) element by element against the
    oracle's operator on the same inputs: G rounded to bfloat16 before the
    oracle sees it (the level's stored geometry), u binary32 values,
    binary64 arithmetic.

    Bound, from the kernel's arithmetic: u, D and the metric's outputs
    (wr, ws) are carried as hi + lo bfloat16 parts, each exact to 2^-17
    relative, and the lo x lo products are dropped, so the operator is off
    by at most about 4 x 2^-17 = 2^-15 of |D|^T |G| |D| |u| at each node,
    plus binary32 accumulation (2^-21 for 16-term sums). The test allows
    2^-14 |A||u|, |A| the operator with |D|, |G|, |B| entry by entry. 18 and
    36 elements: a partial last CTA (four elements per CTA) and full ones."""
    kw = dict(deform_amp=0.05, kappa=KAPPA, phi=PHI)
    om = oracle.box_mesh(nel, 7, **kw)
    gm = sem.sem_mesh_create_box(nel, 7, **kw)
    gp = sem.sem_pmg_create(gm, 1.0, h2, orders=(7, 3, 1), smoother_precision=sem.SEM_PREC_BF16)
    u = np.random.default_rng(9).uniform(-1, 1, om.n_unique).astype(np.float32).astype(np.float64)
    w = torch.empty(om.n_unique, dtype=torch.float64, device="cuda")
    sem.sem_pmg_level_apply(gp, 0, dev(u), w)
    got = host(w)
    Gb = bf16_round(om.G)
    uL = oracle.scatter(om, u * om.mask)
    ref = oracle.gather_sum(om, oracle.ax_local_raw(7, om.D, Gb, om.B, uL, 1.0, h2)) * om.mask
    absA = oracle.gather_sum(om, oracle.ax_local_raw(7, np.abs(om.D), np.abs(Gb), np.abs(om.B), np.abs(uL), 1.0,
                                                     h2)) * om.mask
    err = np.abs(got - ref)
    assert (err <= 2.0 ** -14 * absA).all(), float((err / np.maximum(absA, 1e-300)).max())
    assert (got[om.mask == 0] == 0.0).all()
    gp.destroy()
    gm.destroy()


@pytest.mark.parametrize("h2", [0.0, 3.0], ids=["poisson", "helmholtz"])
def test_bf16_vcycle_matches_oracle_on_bf16_geometry(h2):
    """A bfloat16 V-cycle (tensor-core operator at N = 7, binary32 with
    bfloat16 geometry at N = 3) element by element against the oracle's
    V-cycle run on the same bfloat16-rounded geometry of the smoothing
    levels (lambda_max recomputed from that operator), binary64 arithmetic.
    Bound: a degree-2 V-cycle applies the level-0 operator four times, each
    within 2^-15 of |A||v| (see the operator test), and the Chebyshev-Jacobi
    polynomial is bounded by 1 on the smoother's spectrum: 4 x 2^-15 of
    max|z|."""
    nel = (3, 3, 2)
    box = dict(nel=nel, deform_amp=0.05, kappa=KAPPA, phi=PHI)
    pm = pmg.PMG(box, orders=(7, 3, 1), h2=h2)
    for lev in pm.levels[:-1]:  # the smoothing levels' geometry as the library stores it
        lev.m.G = bf16_round(lev.m.G)
        lev.lam = 1.1 * pm.lambda_max(lev, 20)
    gm = sem.sem_mesh_create_box(nel, 7, deform_amp=0.05, kappa=KAPPA, phi=PHI)
    gp = sem.sem_pmg_create(gm, 1.0, h2, orders=(7, 3, 1), smoother_precision=sem.SEM_PREC_BF16)
    m = pm.levels[0].m
    r = np.random.default_rng(6).standard_normal(m.n_unique) * m.mask
    z = torch.empty(m.n_unique, dtype=torch.float64, device="cuda")
    sem.sem_pmg_vcycle(gp, dev(r), z)
    assert rel_err(host(z), pm.vcycle(r)) < 4 * 2.0 ** -15
    for l in range(2):
        assert abs(gp.lam(l) - pm.levels[l].lam) <= 1e-3 * pm.levels[l].lam
    gp.destroy()
    gm.destroy()


def test_level_apply_arguments():
    """sem_pmg_level_apply: smoothing levels only, no overlapping vectors;
    at a binary32 level it equals the oracle's operator to binary32 accuracy."""
    nel = (2, 2, 2)
    gm = sem.sem_mesh_create_box(nel, 7, deform_amp=0.05, kappa=KAPPA, phi=PHI)
    om = oracle.box_mesh(nel, 7, deform_amp=0.05, kappa=KAPPA, phi=PHI)
    gp = sem.sem_pmg_create(gm, orders=(7, 3, 1))
    u = torch.from_numpy(np.random.default_rng(12).uniform(-1, 1, om.n_unique)).cuda()
    w = torch.empty_like(u)
    for bad in (-1, 2, 3):  # level 2 is the coarsest: no smoother there
        with pytest.raises(sem.SemError) as ei:
            sem.sem_pmg_level_apply(gp, bad, u, w)
        assert ei.value.code == sem.SEM_ERR_INVALID_ARG
    with pytest.raises(sem.SemError):
        sem.sem_pmg_level_apply(gp, 0, u, u)
    sem.sem_pmg_level_apply(gp, 0, u, w)
    ref = oracle.apply_assembled(om, u.cpu().numpy(), 1.0, 0.0)
    assert rel_err(host(w), ref) < 1e-5
    gp.destroy()
    gm.destroy()


def test_bf16_smoother_converges():
    nel, N = (4, 4, 3), 7
    gm = sem.sem_mesh_create_box(nel, N, deform_amp=0.05, kappa=KAPPA, phi=PHI)
    om = oracle.box_mesh(nel, N, deform_amp=0.05, kappa=KAPPA, phi=PHI)
    b = oracle.poisson_rhs(om)
    it = {}
    for name, sp in (("fp32", sem.SEM_PREC_FP32), ("bf16", sem.SEM_PREC_BF16)):
        gp = sem.sem_pmg_create(gm, orders=(7, 3, 1), smoother_precision=sp)
        x = torch.zeros(gm.n_unique, dtype=torch.float64, device="cuda")
        st = sem.sem_pmg_pcg_solve(gp, dev(b), x, tol=1e-8)
        assert st["status"] == 0
        res = np.linalg.norm(b - oracle.apply_assembled(om, host(x))) / np.linalg.norm(b)
        assert res < 1.05e-8
        it[name] = st["iterations"]
        gp.destroy()
    assert it["bf16"] <= 2 * it["fp32"] + 2, it
    gm.destroy()


def test_pmg_invalid_options():
    gm = sem.sem_mesh_create_box((2, 2, 2), 5)
    for kw in (dict(orders=(7, 3)), dict(orders=(5, 5, 1)), dict(orders=(5, 2), smoother_precision=sem.SEM_PREC_FP64),
               dict(orders=(5, 2), smoother_precision=7),
               dict(orders=(5, 2), cheb_degree=0)):
        with pytest.raises(sem.SemError):
            sem.sem_pmg_create(gm, **kw)
    gm.destroy()


def test_neumann_hierarchy_pressure_problem():
    """Pure-Neumann hierarchy (the pressure problem of the time step): the
    mixed solve reaches the tolerance and agrees with Jacobi-PCG up to the
    constant null space."""
    kw = dict(periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), z_stretch=2.0)
    gm = sem.sem_mesh_create_box((4, 4, 4), 7, **kw)
    rng = np.random.default_rng(11)
    b = rng.standard_normal(gm.n_unique)
    b -= b.mean()
    P = sem.sem_pmg_create(gm, orders=(7, 3, 1), mask_mode=1, coarse_tol=1e-2)
    x = torch.zeros(gm.n_unique, dtype=torch.float64, device="cuda")
    st = sem.sem_pmg_pcg_solve(P, dev(b), x, tol=1e-10, mask_mode=1)
    assert st["status"] == 0
    xr = torch.zeros_like(x)
    st2 = sem.sem_pcg_solve(gm, 1.0, 0.0, dev(b), xr, tol=1e-10, maxit=5000, mask_mode=1)
    assert st2["status"] == 0 and st["iterations"] * 5 < st2["iterations"]
    a, c = host(x), host(xr)
    a -= a.mean()
    c -= c.mean()
    assert rel_err(a, c) < 1e-7
    P.destroy()
    gm.destroy()


def test_pmg_48_full_size_solve():
    """The mixed-precision configuration at full size (48^3 elements, N = 7,
    37.9 M unknowns): the p-multigrid flexible CG reaches a true binary64
    relative residual of 1e-8 (checked with the binary64 operator), in both
    smoother precisions."""
    w = workloads.PMG_48
    gm = sem.mesh_from_workload(w)
    u = torch.from_numpy(workloads.unique_field(gm.n_unique, seed=7) * gm.maps()[1]).cuda()
    b = torch.empty_like(u)
    sem.sem_ax_assembled(gm, 1.0, 0.0, u, b, precision=sem.SEM_PREC_FP64)  # b = A u: u is the exact solution
    for sp in (sem.SEM_PREC_FP32, sem.SEM_PREC_BF16):
        P = sem.sem_pmg_create(gm, orders=(7, 3, 1), smoother_precision=sp, coarse_tol=1e-2)
        x = torch.empty_like(u)
        st = sem.sem_pmg_pcg_solve(P, b, x, tol=1e-8)
        assert st["status"] == 0 and st["iterations"] < 40, st
        r = torch.empty_like(u)
        sem.sem_ax_assembled(gm, 1.0, 0.0, x, r, precision=sem.SEM_PREC_FP64)
        assert float(torch.linalg.norm(b - r) / torch.linalg.norm(b)) < 1.2e-8
        assert float((x - u).abs().max() / u.abs().max()) < 1e-3  # error <= condition number x residual
        P.destroy()
    gm.destroy()


@pytest.mark.parametrize("case", range(len(CASES)))
def test_df64_smoothing_matches_the_binary64_oracle(case):
    """The V-cycle with binary64-accurate smoothing (SEM_PREC_DF64: binary64
    level vectors and transfers, double-float operator) against the oracle's
    binary64 V-cycle, both with a tight coarse solve: the eigenvalue bounds,
    the transfers and the whole V-cycle agree to binary64 level."""
    (nel, deform), orders = CASES[case]
    box = dict(nel=nel, deform_amp=deform, kappa=KAPPA, phi=PHI)
    pm = pmg.PMG(box, orders=orders, coarse_tol=1e-13, coarse_maxit=4000)
    gm = sem.sem_mesh_create_box(nel, orders[0], deform_amp=deform, kappa=KAPPA, phi=PHI)
    gp = sem.sem_pmg_create(gm, orders=orders, smoother_precision=sem.SEM_PREC_DF64, coarse_tol=1e-13,
                            coarse_maxit=4000)
    for l in range(len(pm.levels) - 1):
        assert abs(gp.lam(l) - pm.levels[l].lam) <= 1e-10 * pm.levels[l].lam
    rng = np.random.default_rng(8)
    for l in range(len(pm.levels) - 1):
        mf, mc = pm.levels[l].m, pm.levels[l + 1].m
        uc = rng.standard_normal(mc.n_unique) * mc.mask
        uf = torch.empty(mf.n_unique, dtype=torch.float64, device="cuda")
        sem.sem_pmg_prolong(gp, l, dev(uc), uf)
        assert rel_err(host(uf), pm.prolong(l, uc)) < 1e-13
        rf = rng.standard_normal(mf.n_unique) * mf.mask
        rc = torch.empty(mc.n_unique, dtype=torch.float64, device="cuda")
        sem.sem_pmg_restrict(gp, l, dev(rf), rc)
        assert rel_err(host(rc), pm.restrict(l, rf) * mc.mask) < 1e-13
    m = pm.levels[0].m
    r = rng.standard_normal(m.n_unique) * m.mask
    z = torch.empty(m.n_unique, dtype=torch.float64, device="cuda")
    sem.sem_pmg_vcycle(gp, dev(r), z)
    err = rel_err(host(z), pm.vcycle(r))
    assert err < 1e-11, err
    # and as the preconditioner: binary64 residual 1e-8, iterations as the oracle's
    b = oracle.poisson_rhs(m)
    x = torch.zeros(m.n_unique, dtype=torch.float64, device="cuda")
    st = sem.sem_pmg_pcg_solve(gp, dev(b), x, tol=1e-8, maxit=200)
    assert st["status"] == 0
    assert np.linalg.norm(b - oracle.apply_assembled(m, host(x))) / np.linalg.norm(b) < 1.05e-8
    ref = pmg.fcg(pm, b, tol=1e-8)
    assert abs(st["iterations"] - ref.iterations) <= 1, (st, ref.iterations)
    gp.destroy()
    gm.destroy()
