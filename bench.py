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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ax_gs_64")
    ap.add_argument("--no-pcg", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--pcg-tol", type=float, default=1e-8)
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
            "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm
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

    def step():
        sem.sem_ax_assembled(mesh, 1.0, 0.0, u, wg)

    # --- device-resident throughput (the headline value)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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

    # --- kernel-only timing of the dominant kernel (the operator kernel), for the roofline
    dom_ms = ms  # the memset is ~0.1 ms of it; time the kernel through the E-vector entry point too
    uL = torch.empty(mesh.n_local, dtype=torch.float64, device="cuda")
    sem.sem_scatter(mesh, u, uL)
    wL = torch.empty_like(uL)
    for _ in range(3):
        sem.sem_ax_apply(mesh, 1.0, 0.0, uL, wL)
    e0.record(stream)
    for _ in range(args.steps):
        sem.sem_ax_apply(mesh, 1.0, 0.0, uL, wL)
    e1.record(stream)
    torch.cuda.synchronize()
    ax_local_ms = e0.elapsed_time(e1) / args.steps
    # E-vector Ax + gs pair (the unfused form)
    e0.record(stream)
    for _ in range(args.steps):
        sem.sem_ax_apply(mesh, 1.0, 0.0, uL, wL)
        sem.sem_gs_op(mesh, wL, True)
    e1.record(stream)
    torch.cuda.synchronize()
    evec_ms = e0.elapsed_time(e1) / args.steps
    del uL, wL

    flops = FLOP_PER_POINT * w.n_local
    hbm_gbs, hbm_src = peaks()
    achieved_tf = flops / (ax_local_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved_tf / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "k_ax_fp64<8,false> (sem_ax_apply)", "peak_source": "nominal GB300 FP64 rate",
                "hbm_achieved_gbs": BYTES_PER_POINT_AXGS * w.n_local / (dom_ms * 1e-3) / 1e9,
                "hbm_peak_gbs": hbm_gbs, "hbm_peak_source": hbm_src}
    roofline["hbm_frac"] = roofline["hbm_achieved_gbs"] / hbm_gbs

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
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps)
    e2e = {"value": world * w.dofs / (e2e_ms * 1e-3) / 1e9, "unit": "GDOF/s",
           "h2d_bytes_per_step": pin_in.numel() * 8, "d2h_bytes_per_step": pin_out.numel() * 8,
           "ms_per_step": e2e_ms}
    del pin_in, pin_out

    # --- PCG solve time on the same mesh (manufactured-solution right-hand side)
    pcg = None
    if not args.no_pcg:
        # b = M Q^T (B f), f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z), assembled on the device
        # (the forcing at the nodes is input synthesis; the weak form is the library's)
        X, Y, Z = (mesh.field(n) for n in ("X", "Y", "Z"))
        fL = 3.0 * np.pi ** 2 * torch.sin(np.pi * X) * torch.sin(np.pi * Y) * torch.sin(np.pi * Z)
        del X, Y, Z
        b = torch.empty_like(u)
        sem.sem_weak_rhs(mesh, fL, b)
        del fL
        x = torch.zeros_like(u)
        pcg = {}
        for name, prec in (("fp64", sem.SEM_PREC_FP64),):
            torch.cuda.synchronize()
            st = sem.sem_pcg_solve(mesh, 1.0, 0.0, b, x, tol=args.pcg_tol, maxit=20000, precision=prec,
                                   raise_on_error=False)
            pcg[name] = {"iterations": st["iterations"], "solve_ms": st["solve_ms"],
                         "ms_per_iteration": st["solve_ms"] / max(st["iterations"], 1),
                         "rel_residual": st["rel_residual"], "status": st["status"]}
        del b, x

    # --- CPU oracle baseline on rank 0
    cpu = None
    if rank == 0 and not args.no_cpu and world == 1:
        g, cores, sample, _ = time_oracle_axgs(w, 12.0)
        cpu = {"value": g, "unit": "GDOF/s", "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "N": w.N, "nel": list(w.nel), "n_local": w.n_local,
                       "n_unique": w.n_unique, "dofs_per_step": w.dofs, "op": "assembled Ax+gs (Poisson, h1=1)",
                       "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (no flush)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
            "clocks": clocks,
            "extra": {"ax_local_ms": ax_local_ms, "ax_local_gdofs": w.dofs / (ax_local_ms * 1e-3) / 1e9,
                      "evector_ax_plus_gs_ms": evec_ms,
                      "evector_ax_plus_gs_gdofs": w.dofs / (evec_ms * 1e-3) / 1e9, "pcg": pcg},
        }
        print(json.dumps(line))
    mesh.destroy()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
