"""Benchmark of the spectral-element hot path on GB300.

Workload (default ``ax_gs_64``): unit cube of 64^3 hexahedra of order N = 7
(134,217,728 local points, 90,518,849 unique nodes), every GLL node displaced
by the seeded sinusoidal deformation of amplitude 0.1 h, input field
uniform[-1, 1] per unique node (seed 0). Synthetic inputs of the shape of the
paper's p = 7 production meshes (Table "Details of the simulations with
Gamma = 4"); the paper's own meshes and fields are not available.

One step = one application of the assembled operator Ax+gs (w = M Q^T A_L Q M u)
on the whole mesh. ``value`` is GDOF/s in the paper's grid-point convention
(E * N^3 points per application, Sec. 4.4 table). After the timed steps the
same mesh is solved once with Jacobi-PCG to a 1e-8 relative residual (the
"PCG solve time" half of the metric), in every precision the library offers.

Inputs (G alone is 6.4 GB) are far larger than the 129 MB L2, so no flush is
needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "Ax+gs GDOF/s & PCG solve time, FP64 vs mixed at 1e-8 residual; % HBM peak"
FLOP_PER_POINT = 111        # 3 x 2n (D) + 15 (metric) + 3 x 2n (D^T), n = 8
BYTES_PER_POINT_AXGS = 62.7  # G 48 + l2g 4 + (u read + w write) 16 per unique node x 0.674
FP64_PEAK_TFLOPS = 1.25     # GB300 nominal FP64 rate (vector and tensor)
DTYPES = {"df64": "f32x2 (double-float, binary64-accurate)", "fp64": "f64"}
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the assembled
# operator kernel on the 64^3 workload, scaled by points from the ncu capture
# of the 32^3-element case (traffic grows with the points streamed)
TRAFFIC = {"df64": 9.08e9}
# thread instructions per local point of the double-float assembled kernel
# (smsp__inst_executed.sum x 32 / local points, same ncu capture), and the SM
# issue limit: 152 SMs x 4 schedulers x 32 lanes x 2.07 GHz (one warp
# instruction per scheduler per clock)
INST_PER_POINT = {"df64": 491.7}
ISSUE_PEAK_TINST = 152 * 4 * 32 * 2.07e9 / 1e12
# binary32 lane operations per local point of the double-float Poisson operator
# (each packed f32x2 instruction counts two): 6 one-dimensional contractions x
# 59 (even-odd split at N = 7: pair forming 8, 4-term compensated dot products
# 40 per output pair and lane, output pair combination 11 per output), the
# metric 3 x 31, the final three-way sum 19, conversions 3. Peak: the measured
# binary32 FMA rate of this GPU (77 TFLOP/s, own probe) = 38.5 T lane ops/s.
FP32_LANE_OPS_PER_POINT = {"df64": 469.0}
FP32_PEAK_TLANEOPS = 38.5
# Algorithmic bytes of the Rayleigh-Benard step's solves, per unit. Operators
# per local point (E NP^3) plus the gathered/scattered vectors per unique node;
# vector kernels per unique node. Levels of the pressure hierarchy: N = 7, 3, 1.
RBC_UNIT_BYTES = {
    # double-float Helmholtz operator: G 6 x 8 + B 8 + l2g 4 per local point
    "helm_op_local": 60.0,
    # double-float Poisson operator (pressure outer iteration): G 48 + l2g 4
    "poisson_op_local": 52.0,
    # binary32 smoothing operator with bfloat16 geometry: G 6 x 2 + l2g 4
    "smooth_op_local": 16.0,
    # binary64 operand gather and result scatter of an operator, per unique node
    "op_vec64_unique": 16.0,
    "op_vec32_unique": 8.0,
    # Jacobi-PCG iteration vectors: update1 reads x r p w dinv, writes x r;
    # update2 reads r p dinv, writes p w (12 binary64 words)
    "pcg_vec_unique": 96.0,
    # flexible-CG iteration vectors: update with r.r (p w x r read, x r
    # written), binary64<->binary32 at the V-cycle ends (r read, b written;
    # x read, z written), r.zn and r.z, p = zn + beta p with w = 0
    "fcg_vec_unique": 48 + 12 + 12 + 24 + 32,
    # one V-cycle's smoothing vectors on a level at Chebyshev degree 16, in
    # binary32 words: start 5, 15 x (x, d, r, dinv -> x, d) 6, final x += d 3,
    # two residual copies 2 + 2, scaled start 3, 15 x 6, x += d 3, prolongation
    # clear and add 1 + 3
    "cheb_vec_unique_words": 5 + 90 + 3 + 2 + 2 + 3 + 90 + 3 + 1 + 3,
}


def box_counts(w, N):
    """local points and unique nodes of the box workload's mesh at order N"""
    nL = int(np.prod(w.nel)) * (N + 1) ** 3
    nU = int(np.prod([w.nel[d] * N + (0 if w.periodic[d] else 1) for d in range(3)]))
    return nL, nU


def rbc_phase_roofline(w, st, guessed, hbm_gbs):
    """Algorithmic bytes of one Rayleigh-Benard step's three solve phases
    (the per-iteration kernels of each solve; the N = 1 coarse solve of the
    V-cycle is latency-bound and not counted), their rate over the phase's
    measured time and the fraction of the HBM copy rate."""
    b = RBC_UNIT_BYTES
    nL, nU = box_counts(w, w.N)
    helm = nL * b["helm_op_local"] + nU * b["op_vec64_unique"]
    poisson = nL * b["poisson_op_local"] + nU * b["op_vec64_unique"]
    its_u = sum(st["iters_u"])
    g = 1 if guessed else 0  # the operator application that forms r_0 = b - A x0
    out = {}
    out["T"] = (st["iters_T"] + g) * helm + st["iters_T"] * nU * b["pcg_vec_unique"]
    out["u"] = (its_u + 3 * g) * helm + its_u * nU * b["pcg_vec_unique"]
    vc = 0.0
    for N in (w.N, max(1, w.N // 2)):  # smoothing levels 7 and 3
        lL, lU = box_counts(w, N)
        vc += 32 * (lL * b["smooth_op_local"] + lU * b["op_vec32_unique"]) + 4 * lU * b["cheb_vec_unique_words"]
    its_p = st["iters_p"]
    out["p"] = (its_p + g) * poisson + its_p * (nU * b["fcg_vec_unique"] + vc)
    res = {}
    for ph, key in (("T", "ms_T"), ("p", "ms_p"), ("u", "ms_u")):
        gbs = out[ph] / (st[key] * 1e-3) / 1e9 if st[key] > 0 else 0.0
        res[ph] = {"algorithmic_gb": out[ph] / 1e9, "ms": st[key], "achieved_gbs": gbs, "frac": gbs / hbm_gbs}
    tot = sum(out.values())
    ms = st["ms_T"] + st["ms_p"] + st["ms_u"]
    res["solves"] = {"algorithmic_gb": tot / 1e9, "ms": ms, "achieved_gbs": tot / (ms * 1e-3) / 1e9,
                     "frac": tot / (ms * 1e-3) / 1e9 / hbm_gbs}
    return res


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ax_gs_64")
    ap.add_argument("--no-pcg", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-rbc", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--quick-pcg", action="store_true", help="skip the slow binary64 Jacobi-PCG reference solve")
    ap.add_argument("--pcg-tol", type=float, default=1e-8)
    ap.add_argument("--precision", default="df64", choices=["df64", "fp64"])
    ap.add_argument("--once", default="",
                    help="profiling mode: comma list of kernels to launch once each on the workload "
                         "(local_df64, asm_df64, asmh_df64, asmtc1_df64, asmtc2_df64, local_fp64, asm_fp64, gs, vcycle_fp32, vcycle_bf16, pmgsolve_fp32, pmgsolve_bf16, rbc, rbcx, rbcx3, pcg_df64), then exit")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ reference arm
def time_oracle_axgs(w, budget_s: float, max_reps: int = 50):
    """The CPU oracle's assembled operator on a bounded sample of the workload:
    the same mesh construction at a reduced element count (so one application
    takes a fraction of a second), repeated until the time budget is spent."""
    import oracle
    nel_s = 24
    ws = w.with_nel((nel_s, nel_s, nel_s), name=f"{w.name}_sample{nel_s}")
    om = oracle.mesh_from_workload(ws)
    ug = workloads.unique_field(om.n_unique)
    oracle.apply_assembled(om, ug)  # warm-up
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.apply_assembled(om, ug)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= max_reps:
            break
    gdofs = ws.dofs * reps / el / 1e9
    sample = (f"oracle assembled Ax+gs on the {nel_s}^3-element, N={w.N} version of {w.name} "
              f"({ws.n_local} local points), {reps} applications in {el:.1f} s")
    return gdofs, oracle.num_threads(), sample, el / reps


def time_oracle_one_core(w):
    """The same oracle sample on one host core (OpenMP limited to one thread
    in a child process), a few applications."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench, workloads; "
            "g, c, s, _ = bench.time_oracle_axgs(workloads.WORKLOADS[%r], 2.0, max_reps=4); "
            "print(json.dumps({'value': g, 'cores': c, 'sample': s}))") % (ROOT, w.name)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": d["value"], "unit": "GDOF/s", "cores": d["cores"], "sample": d["sample"]}
    except (subprocess.SubprocessError, ValueError, IndexError, KeyError) as e:
        return {"value": None, "note": f"one-core run failed: {type(e).__name__}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workloads.WORKLOADS[args.workload]
    budget = 2.0
    for _ in range(max(args.warmup, 0)):
        time_oracle_axgs(w, 0.0, max_reps=1)
    vals = []
    t_all = 0.0
    for _ in range(max(args.steps, 1)):
        g, cores, sample, per = time_oracle_axgs(w, budget, max_reps=20)
        vals.append(g)
        t_all += per
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / len(vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "N": w.N, "nel": list(w.nel),
                                            "sample": "24^3 elements per step"},
            "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "one_core": time_oracle_one_core(w)},
            "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm
def run_once(sem, mesh, u, names):
    """Launch each named kernel once (for ncu captures of single launches)."""
    import torch
    wg = torch.zeros_like(u)
    uL = torch.empty(mesh.n_local, dtype=torch.float64, device="cuda")
    sem.sem_scatter(mesh, u, uL)
    wL = torch.empty_like(uL)
    P = {"df64": sem.SEM_PREC_DF64, "fp64": sem.SEM_PREC_FP64}
    for name in names:
        kind, _, prec = name.partition("_")
        if kind == "local":
            sem.sem_ax_apply(mesh, 1.0, 0.0, uL, wL, precision=P[prec])
        elif kind == "asm":
            sem.sem_ax_assembled_add(mesh, 1.0, 0.0, u, wg, precision=P[prec])
        elif kind == "asmh":  # the Helmholtz form (h1 = 1, h2 = 0.37)
            sem.sem_ax_assembled_add(mesh, 1.0, 0.37, u, wg, precision=P[prec])
        elif kind in ("asmtc1", "asmtc2"):  # the N = 7 double-float operator on a tensor-core route
            sem.sem_mesh_set_tensor_cores(mesh, 1 if kind == "asmtc1" else 2)
            sem.sem_ax_assembled_add(mesh, 1.0, 0.0, u, wg, precision=P[prec])
            sem.sem_mesh_set_tensor_cores(mesh, 0)
        elif kind == "gs":
            sem.sem_gs_op(mesh, wL, True)
        elif kind in ("rbc", "rbcx", "rbcx3"):  # Rayleigh-Benard steps on the 32^3-element workload
            rw = workloads.RBC_32
            rm = sem.mesh_from_workload(rw)
            pert = torch.from_numpy(workloads.perturbation(rm.n_unique, 1e-3)).cuda()
            # rbcx: solves from the extrapolated guess, four steps (the fourth steady);
            # rbcx3: the same with third-order guesses for the temperature and velocity
            rs = sem.sem_rbc_create(rm, 1e8, 0.7, 1e-3, tol=1e-8, precision=sem.SEM_PREC_DF64, T_pert=pert,
                                    extrapolate={"rbc": 0, "rbcx": 1, "rbcx3": 2}[kind])
            for _ in range(3 if kind == "rbc" else 4):
                print(json.dumps(sem.sem_bdf_ext_step(rs)))
            rs.destroy()
            rm.destroy()
        elif kind == "pcg":  # 16 Jacobi-PCG iterations (no stopping), for launch lists
            b = torch.ones_like(u)
            x = torch.zeros_like(u)
            st = sem.sem_pcg_solve(mesh, 1.0, 0.0, b, x, tol=0.0, maxit=16, precision=P[prec],
                                   raise_on_error=False)
            print(json.dumps(st))
        elif kind == "pmgsolve":  # 4 p-multigrid flexible-CG iterations (no stopping), for launch lists
            sp = {"fp32": sem.SEM_PREC_FP32, "bf16": sem.SEM_PREC_BF16}[prec]
            H = sem.sem_pmg_create(mesh, orders=(mesh.N, 3, 1), smoother_precision=sp, coarse_tol=1e-2)
            b = torch.ones_like(u)
            x = torch.zeros_like(u)
            st = sem.sem_pmg_pcg_solve(H, b, x, tol=0.0, maxit=4, raise_on_error=False)
            print(json.dumps(st))
            H.destroy()
        elif kind == "vcycle":
            sp = {"fp32": sem.SEM_PREC_FP32, "bf16": sem.SEM_PREC_BF16}[prec]
            H = sem.sem_pmg_create(mesh, orders=(mesh.N, 3, 1), smoother_precision=sp, coarse_tol=1e-2)
            z = torch.empty_like(u)
            sem.sem_pmg_vcycle(H, u, z)
            torch.cuda.synchronize()
            H.destroy()
        else:
            raise ValueError(name)
    torch.cuda.synchronize()
    print(json.dumps({"once": names, "workload": "ok"}))
    return 0


def run_solves(sem, mesh, w, runs, tol):
    """Solve the manufactured Poisson problem on `mesh` with each listed
    solver to `tol`; iterations, times, true binary64 residuals and the
    difference to the first (reference) solution."""
    import torch
    # (the forcing at the nodes is input synthesis; the weak form is the library's)
    X, Y, Z = (mesh.field(n) for n in ("X", "Y", "Z"))
    fL = 3.0 * np.pi ** 2 * torch.sin(np.pi * X) * torch.sin(np.pi * Y) * torch.sin(np.pi * Z)
    del X, Y, Z
    b = torch.empty(mesh.n_unique, dtype=torch.float64, device="cuda")
    sem.sem_weak_rhs(mesh, fL, b)
    del fL
    out, sols = {}, {}
    for name, kind, prec, sprec in runs:
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        setup_ms = 0.0
        if kind == "jacobi":
            st = sem.sem_pcg_solve(mesh, 1.0, 0.0, b, x, tol=tol, maxit=20000, precision=prec, raise_on_error=False)
        else:
            t0 = time.perf_counter()
            # the configuration's degree-2 Chebyshev smoothing ("pmg"), and degree 3 beside it ("pmg3")
            P = sem.sem_pmg_create(mesh, orders=(w.N, 3, 1) if w.N > 3 else (w.N, 1), smoother_precision=sprec,
                                   coarse_tol=1e-2, cheb_degree=3 if kind == "pmg3" else 2)
            setup_ms = 1e3 * (time.perf_counter() - t0)
            st = sem.sem_pmg_pcg_solve(P, b, x, tol=tol, maxit=500, precision=prec, raise_on_error=False)
            # one V-cycle on its own (CUDA events, 5 after one warm-up)
            z = torch.empty_like(b)
            sem.sem_pmg_vcycle(P, b, z)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record()
            for _ in range(5):
                sem.sem_pmg_vcycle(P, b, z)
            ev1.record()
            torch.cuda.synchronize()
            vcycle_ms = ev0.elapsed_time(ev1) / 5
            del z
            P.destroy()
        rr = torch.empty_like(b)  # true residual with the binary64 operator
        sem.sem_ax_assembled(mesh, 1.0, 0.0, x, rr, precision=sem.SEM_PREC_FP64)
        true_res = float(torch.linalg.norm(b - rr) / torch.linalg.norm(b))
        if kind == "jacobi":
            vcycle_ms = None
        out[name] = {"iterations": st["iterations"], "solve_ms": st["solve_ms"], "setup_ms": setup_ms,
                     "vcycle_ms": vcycle_ms,
                     "ms_per_iteration": st["solve_ms"] / max(st["iterations"], 1),
                     "rel_residual": st["rel_residual"], "true_rel_residual_fp64": true_res, "status": st["status"]}
        sols[name] = x
    ref_name = runs[0][0]
    ref = sols[ref_name]
    for name, x in sols.items():
        out[name]["solution_rel_diff_vs_" + ref_name] = float((x - ref).abs().max() / ref.abs().max())
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_2501_13240_gb300 as sem

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        # replicas: the scaling run measures the headline step only (the
        # solver, RBC, adjoint and rendering sections are single-GPU reports)
        args.no_pcg = args.no_rbc = args.no_adjoint = True

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    w = workloads.WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    mesh = sem.mesh_from_workload(w)
    ug_host = workloads.unique_field(mesh.n_unique)
    u = torch.from_numpy(ug_host).cuda()
    wg = torch.empty_like(u)
    if args.once:
        return run_once(sem, mesh, u, args.once.split(","))
    precs = {"df64": sem.SEM_PREC_DF64, "fp64": sem.SEM_PREC_FP64}
    head = args.precision
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step(prec=precs[head]):
        sem.sem_ax_assembled(mesh, 1.0, 0.0, u, wg, precision=prec)

    def timed(fn, n):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    # --- device-resident throughput (the headline value)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms)
    value = world * w.dofs / (ms * 1e-3) / 1e9
    clocks = clk.summary()

    # --- per-precision timings: assembled op, its kernel alone (accumulating
    # entry point, no clearing of w), and the E-vector Ax + gs pair
    uL = torch.empty(mesh.n_local, dtype=torch.float64, device="cuda")
    sem.sem_scatter(mesh, u, uL)
    wL = torch.empty_like(uL)
    nrep = max(3, min(args.steps, 10))
    per = {}
    for name, prec in precs.items():
        per[name] = {
            "assembled_ms": timed(lambda: step(prec), nrep),
            "kernel_ms": timed(lambda: sem.sem_ax_assembled_add(mesh, 1.0, 0.0, u, wg, precision=prec), nrep),
            "ax_local_ms": timed(lambda: sem.sem_ax_apply(mesh, 1.0, 0.0, uL, wL, precision=prec), nrep),
            "evector_ax_gs_ms": timed(lambda: (sem.sem_ax_apply(mesh, 1.0, 0.0, uL, wL, precision=prec),
                                               sem.sem_gs_op(mesh, wL, True)), nrep),
        }
        per[name]["assembled_gdofs"] = w.dofs / (per[name]["assembled_ms"] * 1e-3) / 1e9
    del uL, wL

    hbm_gbs, hbm_src = peaks()
    kms = per[head]["kernel_ms"]
    algo_bytes = BYTES_PER_POINT_AXGS * w.n_local
    achieved = algo_bytes / (kms * 1e-3) / 1e9
    fp64_tf = FLOP_PER_POINT * w.n_local / (per["fp64"]["kernel_ms"] * 1e-3) / 1e12
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s", "frac": achieved / hbm_gbs,
                "traffic": TRAFFIC.get(head), "kernel": f"k_ax_{head}<8, assembled>",
                "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": algo_bytes, "kernel_ms": kms,
                "fp64_kernel": {"bound": "alu", "achieved_tflops": fp64_tf, "peak_tflops": FP64_PEAK_TFLOPS,
                                "frac": fp64_tf / FP64_PEAK_TFLOPS, "peak_source": "nominal GB300 FP64 rate"}}
    if head in INST_PER_POINT:  # what actually binds the double-float kernel: instruction issue
        ti = INST_PER_POINT[head] * w.n_local / (kms * 1e-3) / 1e12
        roofline["issue_view"] = {"bound": "alu", "achieved_tinst_per_s": ti, "peak_tinst_per_s": ISSUE_PEAK_TINST,
                                  "frac": ti / ISSUE_PEAK_TINST,
                                  "peak_source": "152 SMs x 4 schedulers x 32 lanes x 2.07 GHz",
                                  "inst_per_point_source": "ncu smsp__inst_executed.sum, ax_gs_32"}
    if head in FP32_LANE_OPS_PER_POINT:  # ... and the binary32 pipe it computes on
        tl = FP32_LANE_OPS_PER_POINT[head] * w.n_local / (kms * 1e-3) / 1e12
        roofline["fp32_pipe_view"] = {"bound": "alu", "achieved_tlaneops_per_s": tl,
                                      "peak_tlaneops_per_s": FP32_PEAK_TLANEOPS, "frac": tl / FP32_PEAK_TLANEOPS,
                                      "peak_source": "measured binary32 FMA rate (own probe, 77 TFLOP/s)",
                                      "lane_ops_per_point": FP32_LANE_OPS_PER_POINT[head]}

    # --- end to end through the C ABI with host buffers
    pin_in = torch.from_numpy(ug_host).pin_memory()
    pin_out = torch.empty(mesh.n_unique, dtype=torch.float64).pin_memory()
    for _ in range(2):
        u.copy_(pin_in, non_blocking=True)
        step()
        pin_out.copy_(wg, non_blocking=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    e2e_steps = max(3, args.steps // 3)
    for _ in range(e2e_steps):
        u.copy_(pin_in, non_blocking=True)
        step()
        pin_out.copy_(wg, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    serial_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps)
    # the library's host-buffer entry point: the same operator with the
    # copies pipelined against the arithmetic in z-slabs (the timed call
    # includes every host<->device byte of the step)
    prec_code = {"df64": sem.SEM_PREC_DF64, "fp64": sem.SEM_PREC_FP64}[head]
    for _ in range(2):
        sem.sem_ax_assembled_host(mesh, 1.0, 0.0, pin_in, pin_out, u, wg, prec_code)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    for _ in range(e2e_steps):
        sem.sem_ax_assembled_host(mesh, 1.0, 0.0, pin_in, pin_out, u, wg, prec_code)
    e1.record(stream)
    torch.cuda.synchronize()
    call_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps)
    # the batched entry point: the same steps pipelined across each other
    # (copy-in of step k + 1, operator of step k, copy-out of step k - 1), one
    # whole-vector copy each way per step, device vectors double-buffered
    pin_outs = [pin_out, torch.empty(mesh.n_unique, dtype=torch.float64).pin_memory()]
    u2 = torch.empty(2 * mesh.n_unique, dtype=torch.float64, device=u.device)
    w2 = torch.empty_like(u2)
    sem.sem_ax_assembled_host_batch(mesh, 1.0, 0.0, [pin_in] * 2, pin_outs, u2, w2, prec_code)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)  # exactly K steps, like the headline
    sem.sem_ax_assembled_host_batch(mesh, 1.0, 0.0, [pin_in] * args.steps,
                                    [pin_outs[k % 2] for k in range(args.steps)], u2, w2, prec_code)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    e2e = {"value": world * w.dofs / (e2e_ms * 1e-3) / 1e9, "unit": "GDOF/s",
           "h2d_bytes_per_step": pin_in.numel() * 8, "d2h_bytes_per_step": pin_out.numel() * 8,
           "ms_per_step": e2e_ms,
           "call": f"sem_ax_assembled_host_batch ({args.steps} steps in one call, pinned host vectors)",
           "per_call_value": world * w.dofs / (call_ms * 1e-3) / 1e9, "per_call_ms": call_ms,
           "per_call": "sem_ax_assembled_host (one step per call, 8 z-slabs)",
           "serialised_copy_step_copy_ms": serial_ms,
           "serialised_value": world * w.dofs / (serial_ms * 1e-3) / 1e9}
    del pin_in, pin_out, pin_outs, u2, w2

    # --- solve time on the same mesh (manufactured forcing): binary64 Jacobi-PCG
    # against the mixed-precision p-multigrid flexible CG, all to 1e-8
    pcg = None
    if not args.no_pcg:
        runs = [("jacobi_fp64", "jacobi", sem.SEM_PREC_FP64, None),
                ("jacobi_df64", "jacobi", sem.SEM_PREC_DF64, None),
                ("pmg_fp32_df64", "pmg", sem.SEM_PREC_DF64, sem.SEM_PREC_FP32),
                ("pmg_bf16_df64", "pmg", sem.SEM_PREC_DF64, sem.SEM_PREC_BF16),
                ("pmg_df64_df64", "pmg", sem.SEM_PREC_DF64, sem.SEM_PREC_DF64),
                ("pmg_fp32_df64_cheb3", "pmg3", sem.SEM_PREC_DF64, sem.SEM_PREC_FP32)]
        if args.quick_pcg:
            runs = [r for r in runs if r[0] != "jacobi_fp64"]
        pcg = run_solves(sem, mesh, w, runs, args.pcg_tol)
    # the mixed-precision configuration on its own mesh: the 64^3 construction
    # at 48^3 elements (37.9 M unknowns); reference = double-float Jacobi-PCG
    pcg48 = None
    if not args.no_pcg:
        w48 = workloads.PMG_48
        m48 = sem.mesh_from_workload(w48)
        pcg48 = run_solves(sem, m48, w48, [("jacobi_df64", "jacobi", sem.SEM_PREC_DF64, None),
                                           ("pmg_fp32_df64", "pmg", sem.SEM_PREC_DF64, sem.SEM_PREC_FP32),
                                           ("pmg_bf16_df64", "pmg", sem.SEM_PREC_DF64, sem.SEM_PREC_BF16),
                                           ("pmg_df64_df64", "pmg", sem.SEM_PREC_DF64, sem.SEM_PREC_DF64),
                                           ("pmg_fp32_df64_cheb3", "pmg3", sem.SEM_PREC_DF64, sem.SEM_PREC_FP32)],
                           args.pcg_tol)
        pcg48["workload"] = w48.name
        m48.destroy()

    # --- Rayleigh-Benard BDF2/EXT2 steps (32^3 elements, Ra = 1e8, Pr = 0.7),
    # solves from zero, from the extrapolated guess 2 x^n - x^{n-1}, and with
    # the temperature and velocity from 3 x^n - 3 x^{n-1} + x^{n-2}
    rbc = None
    if not args.no_rbc:
        rw = workloads.RBC_32
        rm = sem.mesh_from_workload(rw)
        pert = torch.from_numpy(workloads.perturbation(rm.n_unique, 1e-3)).cuda()
        hbm_gbs, _ = peaks()
        rbc = {"workload": rw.name, "tol": 1e-8, "unit_bytes": RBC_UNIT_BYTES,
               "roofline_peak_gbs": hbm_gbs}
        keep = None
        for mode, ex in (("cold", 0), ("extrapolated", 1), ("extrapolated3", 2)):
            rs = sem.sem_rbc_create(rm, 1e8, 0.7, 1e-3, tol=1e-8, precision=sem.SEM_PREC_DF64, T_pert=pert,
                                    extrapolate=ex)
            steps = [sem.sem_bdf_ext_step(rs, raise_on_error=False) for _ in range(5)]
            for s_ in steps:
                s_["phase_roofline"] = rbc_phase_roofline(rw, s_, bool(ex) and s_["step"] > 1, hbm_gbs)
            rbc[mode] = {"steps": steps,
                         "ms_per_step_after_first": float(np.mean([s_["step_ms"] for s_ in steps[1:]])),
                         # the first two steps differ (BDF1, then new Jacobi inverses for b0 = 3/2);
                         # step times are host wall clock, so the median is also given
                         "ms_per_steady_step": float(np.mean([s_["step_ms"] for s_ in steps[2:]])),
                         "ms_per_steady_step_median": float(np.median([s_["step_ms"] for s_ in steps[2:]]))}
            if mode == "extrapolated":  # its temperature is rendered below
                keep = rs
                T = sem.sem_rbc_fields(rs)["T"]
            else:
                rs.destroy()
        # in-situ rendering of the temperature: bottom boundary-layer slice and a
        # vertical slice, 4096 x 4096 pixels each, iso-levels 0.4 and 0.6
        render = {}
        for name, axis, coord in (("bottom_bl_z0.01", 2, 0.01), ("vertical_y0.5", 1, 0.5)):
            vals = torch.empty((4096, 4096), dtype=torch.float32, device="cuda")
            rgba = torch.empty((4096, 4096, 4), dtype=torch.uint8, device="cuda")
            for _ in range(2):
                sem.sem_render_slice(rm, T, axis, coord, 4096, 4096, 0.0, 1.0, (0.4, 0.6), vals, rgba)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(5):
                sem.sem_render_slice(rm, T, axis, coord, 4096, 4096, 0.0, 1.0, (0.4, 0.6), vals, rgba)
            rms = 1e3 * (time.perf_counter() - t0) / 5
            render[name] = {"ms": rms, "mpixel_per_s": 4096 * 4096 / (rms * 1e-3) / 1e6}
            del vals, rgba
        # the overview scene: iso-surfaces 0.4 and 0.6 in perspective, 4096 x 2048
        # pixels, field resampled to 256^3
        sv = torch.empty((256, 256, 256), dtype=torch.float32, device="cuda")
        sd = torch.empty((2048, 4096), dtype=torch.float32, device="cuda")
        sr = torch.empty((2048, 4096, 4), dtype=torch.uint8, device="cuda")
        cam = ((2.2, -1.6, 1.6), (0.5, 0.5, 0.45), (0.0, 0.0, 1.0), 35.0)
        for _ in range(2):
            sem.sem_render_scene(rm, T, *cam, 4096, 2048, (256, 256, 256), 0.0, 1.0, (0.4, 0.6), sv, sd, sr)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            sem.sem_render_scene(rm, T, *cam, 4096, 2048, (256, 256, 256), 0.0, 1.0, (0.4, 0.6), sv, sd, sr)
        rms = 1e3 * (time.perf_counter() - t0) / 3
        render["iso_scene_4096x2048_grid256"] = {"ms": rms, "hit_fraction": float((sd >= 0).float().mean())}
        del sv, sd, sr
        rbc["render_4096x4096"] = render
        keep.destroy()
        rm.destroy()

    # --- adjoint: gradient of the bottom-plate Nusselt number after K = 20
    # steps with respect to T^0 (16^3 elements, N = 7, Ra = 1e7, Pr = 1),
    # velocity history checkpointed every 5 steps; deterministic assembly so
    # that replayed segments equal the original run bit for bit
    adj = None
    if not args.no_adjoint:
        from paper_2501_13240_gb300 import adjoint as gadj
        aw = workloads.ADJOINT_16
        am = sem.mesh_from_workload(aw, deterministic=True)
        Ra, Pr, dt, K = 1e7, 1.0, 2e-3, 20
        pert = torch.from_numpy(workloads.perturbation(am.n_unique, 1e-2, seed=2)).cuda()
        rs = sem.sem_rbc_create(am, Ra, Pr, dt, tol=1e-10, precision=sem.SEM_PREC_DF64, T_pert=pert)
        T0 = sem.sem_rbc_fields(rs)["T"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist = gadj.VelocityHistory(rs, K, 5)
        torch.cuda.synchronize()
        run_ms = 1e3 * (time.perf_counter() - t0)
        ta = sem.sem_tadv_create(am, 1.0 / np.sqrt(Ra * Pr), dt, tol=1e-13, precision=sem.SEM_PREC_DF64)
        x = T0.clone().requires_grad_(True)
        t0 = time.perf_counter()
        nu = gadj.nusselt_after(x, hist, ta)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        nu.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        mask = torch.from_numpy(am.maps()[1].astype(np.float64)).cuda()
        rng = np.random.default_rng(31)
        fd_err = []
        for _ in range(2):
            d = torch.from_numpy(rng.standard_normal(am.n_unique)).cuda() * mask
            fp = float(gadj.nusselt_after(T0 + 1e-6 * d, hist, ta))
            fm = float(gadj.nusselt_after(T0 - 1e-6 * d, hist, ta))
            fd = (fp - fm) / 2e-6
            fd_err.append(abs(fd - float(torch.dot(x.grad, d))) / abs(fd))
        adj = {"workload": aw.name, "K": K, "checkpoint_every": 5, "Nu_b": float(nu.detach()),
               "rbc_run_ms": run_ms, "forward_ms": 1e3 * (t1 - t0), "backward_ms": 1e3 * (t2 - t1),
               "rbc_steps_replayed": hist.n_replayed, "fd_rel_err_2_directions": fd_err}
        del hist, x, T0
        ta.destroy()
        rs.destroy()
        am.destroy()

    # --- CPU oracle baseline on rank 0
    cpu = None
    if rank == 0 and not args.no_cpu and world == 1:
        g, cores, sample, _ = time_oracle_axgs(w, 12.0)
        cpu = {"value": g, "unit": "GDOF/s", "cores": cores, "kind": "oracle", "sample": sample,
               "one_core": time_oracle_one_core(w)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES[head], "data": "synthetic",
            "config": {"workload": w.name, "N": w.N, "nel": list(w.nel), "n_local": w.n_local,
                       "n_unique": w.n_unique, "dofs_per_step": w.dofs, "op": "assembled Ax+gs (Poisson, h1=1)",
                       "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (no flush)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
            "clocks": clocks,
            "extra": {"precision": head, "per_precision": per, "solves": pcg, "solves_pmg_48": pcg48, "rbc_step": rbc,
                      "adjoint": adj},
        }
        print(json.dumps(line))
    mesh.destroy()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
