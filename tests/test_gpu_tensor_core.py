"""GPU parity of the N = 7 double-float operator whose 1-D contractions run
exactly on the fp16 tensor cores (digit slicing, Sec. 2.2's dense tensor
contractions), against the FP64 oracle and against the binary32-pipe route,
through the C ABI. Routes: 1 (four warps per element through shared
memory), 2 (one warp per element in registers; Poisson calls with the masked
map, others fall back to route 0) and 0 (the binary32 pipe). Tolerance: the FP64 parity bar, 1e-12 relative in the max
norm. Edge cases: inputs whose digits sit at the ends of their range, a
constant field (cancellation in every contraction), elements mixing values
30 orders of magnitude apart, zero and impulse inputs, NaN."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import paper_2501_13240_gb300 as sem  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL = 1e-12
KAPPA = np.array([[1.0, 2.0, 1.0], [2.0, 1.0, 1.0], [1.0, 1.0, 2.0]])
PHI = np.array([0.3, 1.7, 4.1])
DF = sem.SEM_PREC_DF64

SPECS = [
    dict(nel=(5, 3, 3), deform_amp=0.05),  # 45 elements, deformed: all six G factors vary
    dict(nel=(2, 3, 4), deform_amp=0.04, periodic=(1, 1, 0), dirichlet=(0, 0, 0, 0, 1, 1), z_stretch=2.0,
         L=(1.0, 1.0, 1.0)),
    dict(nel=(3, 2, 2), deform_amp=0.0, L=(2.0, 1.0, 0.5)),
]


def rel_err(a, b):
    s = np.abs(b).max()
    return np.abs(np.asarray(a) - b).max() / (s if s > 0 else 1.0)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def make(spec):
    kw = dict(N=7, kappa=KAPPA, phi=PHI, **spec)
    om = oracle.box_mesh(spec["nel"], 7, spec.get("L", (1.0, 1.0, 1.0)), spec.get("periodic", (0, 0, 0)),
                         spec.get("dirichlet", (1,) * 6), spec.get("z_stretch", 0.0), spec["deform_amp"], KAPPA, PHI)
    return om, sem.sem_mesh_create_box(**kw)


@pytest.fixture(scope="module", params=range(len(SPECS)), ids=lambda i: "mesh%d" % i)
def pair(request):
    om, gm = make(SPECS[request.param])
    yield om, gm
    gm.destroy()


ROUTES = (1, 2, 0)


def both_routes(gm, fn):
    """fn() with each route: the two tensor-core routes, then the binary32 route (the default)"""
    out = []
    for on in ROUTES:
        sem.sem_mesh_set_tensor_cores(gm, on)
        out.append(fn())
    return out


@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.37, 12.5), (0.0, 2.0)])
def test_local_operator_both_routes(pair, h1, h2):
    om, gm = pair
    u = np.random.default_rng(31).uniform(-1, 1, om.n_local)
    ref = oracle.ax_local(om, u, h1, h2)

    def run():
        w = torch.empty(om.n_local, dtype=torch.float64, device="cuda")
        sem.sem_ax_apply(gm, h1, h2, dev(u), w, precision=DF)
        return host(w)

    for got in both_routes(gm, run):
        assert rel_err(got, ref) < RTOL


@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.37, 12.5)])
@pytest.mark.parametrize("deterministic", [False, True])
def test_assembled_operator_both_routes(pair, h1, h2, deterministic):
    om, gm = pair
    ug = np.random.default_rng(32).uniform(-1, 1, om.n_unique)
    ref = oracle.apply_assembled(om, ug, h1, h2)
    sem.sem_mesh_set_deterministic(gm, deterministic)

    def run():
        w = torch.empty(om.n_unique, dtype=torch.float64, device="cuda")
        sem.sem_ax_assembled(gm, h1, h2, dev(ug), w, precision=DF)
        return host(w)

    first = both_routes(gm, run)
    sem.sem_mesh_set_deterministic(gm, False)
    for got in first:
        assert rel_err(got, ref) < RTOL
    if deterministic:  # fixed-order assembly repeats bit for bit, on every route
        sem.sem_mesh_set_deterministic(gm, True)
        again = both_routes(gm, run)
        sem.sem_mesh_set_deterministic(gm, False)
        for a, b in zip(again, first):
            np.testing.assert_array_equal(a, b)


def input_cases(om):
    rng = np.random.default_rng(33)
    n = om.n_local
    yield "digit_edges", np.where(rng.random(n) < 0.5, 1.0, -1.0) * (1.0 - 2.0 ** -53) * rng.choice(
        [1.0, 0.5, 0.75, 2.0 ** -10, 1.0 - 2.0 ** -11], n)
    yield "constant", np.full(n, 0.7) + 1e-9 * rng.standard_normal(n)
    mixed = rng.uniform(-1, 1, n)
    mixed[rng.random(n) < 0.5] *= 1e-30
    yield "mixed_magnitudes", mixed
    yield "zero", np.zeros(n)
    imp = np.zeros(n)
    imp[rng.integers(0, n, 3)] = [1.0, -3.0, 2.5e-7]
    yield "impulses", imp
    yield "huge", rng.uniform(-1, 1, n) * 1e280


@pytest.mark.parametrize("tc", ROUTES, ids=["tensor", "tensor_registers", "binary32"])
@pytest.mark.parametrize("case", ["digit_edges", "constant", "mixed_magnitudes", "zero", "impulses", "huge"])
def test_edge_inputs(case, tc):
    om, gm = make(SPECS[0])
    sem.sem_mesh_set_tensor_cores(gm, tc)
    u = dict(input_cases(om))[case]
    h1, h2 = (1.0, 0.0) if tc == 2 else (0.37, 12.5)  # route 2 takes the Poisson operator
    ref = oracle.ax_local(om, u, h1, h2)
    w = torch.empty(om.n_local, dtype=torch.float64, device="cuda")
    sem.sem_ax_apply(gm, h1, h2, dev(u), w, precision=DF)
    got = host(w)
    assert np.isfinite(got).all()
    if case == "zero":
        assert (got == 0.0).all()
    else:
        # relative to the operator's scale |A||u| = |D|^T |G| |D| |u| (+ h2 B
        # |u|), entry by entry (the constant field cancels almost exactly, so
        # not relative to |Au|)
        absA = oracle.ax_local_raw(om.N, np.abs(om.D), np.abs(om.G), np.abs(om.B), np.abs(u), h1, h2)
        if case == "constant":  # A u cancels to ~1e-9 of |A||u|: the parity bar is taken against |A||u|
            scale = np.abs(absA).max()
        else:
            scale = max(np.abs(ref).max(), 1e-3 * np.abs(absA).max())
        assert np.abs(got - ref).max() < RTOL * scale, case
    gm.destroy()


@pytest.mark.parametrize("tc", ROUTES, ids=["tensor", "tensor_registers", "binary32"])
def test_nan_propagates_to_breakdown(tc):
    gm = sem.sem_mesh_create_box((3, 2, 2), 7)
    sem.sem_mesh_set_tensor_cores(gm, tc)
    b = torch.zeros(gm.n_unique, dtype=torch.float64, device="cuda")
    b[gm.n_unique // 2] = float("nan")
    st = sem.sem_pcg_solve(gm, 1.0, 0.0, b, torch.zeros_like(b), precision=DF, raise_on_error=False)
    assert st["status"] == sem.SEM_ERR_BREAKDOWN
    gm.destroy()


@pytest.mark.parametrize("h1,h2", [(0.5, 40.0), (1.0, 0.0)], ids=["helmholtz", "poisson"])
def test_pcg_iterations_match_oracle_on_both_routes(pair, h1, h2):
    """Jacobi-PCG on every route: the iterations of the oracle (+-1) and its
    solution; on route 2 the Poisson solve's p.w comes from the energy form
    sum (ur wr + us ws + ut wt) of each element."""
    om, gm = pair
    if h2 == 0.0 and om.mask.sum() == om.n_unique:
        pytest.skip("singular without Dirichlet nodes")
    b = np.random.default_rng(34).standard_normal(om.n_unique) * om.mask
    ref = oracle.pcg(om, b, h1, h2, tol=1e-10, maxit=3000)

    def run():
        x = torch.zeros(om.n_unique, dtype=torch.float64, device="cuda")
        st = sem.sem_pcg_solve(gm, h1, h2, dev(b), x, tol=1e-10, maxit=3000, precision=DF)
        return st, host(x)

    for st, x in both_routes(gm, run):
        assert st["status"] == 0 and abs(st["iterations"] - ref.iterations) <= 1
        assert rel_err(x, ref.x) < 1e-9
