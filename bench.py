#!/usr/bin/env python
"""Benchmark of the Wilson-Dirac hot path on one GB300 (or N replicas).

Metric: dslash GB/s against the HBM peak, and the wall time of the
reliable-update mixed-precision solve to |b - M x|/|b| <= 1e-12 against the
pure FP64 solve on the same lattice (arXiv:0911.3191, Sec. 4-5).

A step is one whole solve of the workload (24^3 x 64 lattice, SU(3) links
exp(0.3 i H), kappa = 0.124, complex-Gaussian source, even-odd BiCGstab with a
16-bit (Q16) inner iteration and FP64 reliable updates, delta = 0.1, tol
1e-12): Schur source, iteration, reliable updates, reconstruction and the FP64
true residual all run inside the step.  `value` is solves per second with
the inputs resident in HBM; `e2e` is the same through wd_solve with host
buffers (host->device source, device->host solution inside the timing).

Multi-GPU: the solve does not shard here, so N ranks run N independent
replicas (weak scaling) with a barrier and max-over-ranks timing.

--impl reference times the FP64 CPU oracle (the deliberately slow checker)
on a bounded sample of the same solve.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {
    "workload": "wilson-dirac even-odd BiCGstab 24^3x64, eps=0.3, kappa=0.124, tol=1e-12, "
                "inner=q16 + fp64 reliable updates (delta=0.1)",
    "dims": (24, 24, 24, 64), "eps": 0.3, "kappa": 0.124, "tol": 1e-12, "delta": 0.1,
    "gauge_seed": 1001, "source_seed": 2001,
}
METRIC = "dslash GB/s vs HBM peak; mixed vs FP64 solve time to |r|/|b|<=1e-12"
# algorithmic bytes per output site of one dslash, 12-real links: 8 links,
# one input spinor, one output spinor (each link and input read once)
BYTES_PER_SITE = {0: 8 * 96 + 192 + 192, 1: 8 * 48 + 96 + 96, 2: 8 * 24 + 52 + 52, 3: 8 * 24 + 52 + 52,
                  4: 8 * 24 + 52 + 52}
FLOPS_PER_SITE = 1320  # the paper's effective count (Sec. 4.3)
PREC_NAME = {0: "f64", 1: "f32", 2: "q16", 3: "h16n", 4: "b16n"}
ORACLE_ITERS = os.path.join(ROOT, "tests", "golden", "oracle_fp64_iterations.json")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_iterations(kappa: float) -> int:
    with open(ORACLE_ITERS) as f:
        d = json.load(f)
    return int(d["bicgstab_schur"][f"{kappa:.3f}"]["iterations"])


def cpu_baseline(U, b, dims, kappa, iters_full: int, sample_iters: int):
    """The oracle as it stands: FP64 BiCGstab on the Schur system, a bounded
    sample of iterations, scaled to a full solve of iters_full iterations."""
    import oracle
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    oracle._load()
    t0 = time.perf_counter()
    oracle.bicgstab_schur_iterations(b, U, dims, kappa, sample_iters)
    dt = time.perf_counter() - t0
    per_solve = dt / sample_iters * iters_full
    return {"value": 1.0 / per_solve, "unit": "solves/s", "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle",
            "sample": f"{sample_iters} FP64 BiCGstab iterations of the {dims[0]}^3x{dims[3]} Schur solve "
                      f"({dt:.1f} s), scaled to the {iters_full} iterations of the full FP64 solve"}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import lattice_inputs as li
    W = WORKLOAD
    dims, kappa = W["dims"], W["kappa"]
    U = li.gauge(dims, W["eps"], W["gauge_seed"])
    b = li.gaussian_spinor(dims, W["source_seed"])
    iters_full = oracle_iterations(kappa)
    sample = 6
    for _ in range(args.warmup):
        cpu_baseline(U, b, dims, kappa, iters_full, 2)
    vals = [cpu_baseline(U, b, dims, kappa, iters_full, sample) for _ in range(args.steps)]
    v = statistics.mean(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["workload"], "lattice": "24x24x24x64"},
            "cpu_baseline": {**vals[0], "value": v},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def time_dslash(wd, torch, prec, n, flush=None):
    """Average device time of one dslash launch (CUDA events on the
    library's stream), optionally flushing L2 between launches."""
    import paper_0911_3191_gb300 as wdp
    fin = wd.new_field(prec)
    fout = wd.new_field(prec)
    fin.zero_()
    s = wd.stream
    for _ in range(3):
        wd.dslash(fout, fin, wdp.EVEN, False, prec)
    ts = []
    for _ in range(n):
        if flush is not None:
            flush.add_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        wd.dslash(fout, fin, wdp.EVEN, False, prec)
        e1.record(s)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1000.0)
    return statistics.mean(ts)


def run_ours(args):
    import numpy as np
    import torch

    import lattice_inputs as li
    import paper_0911_3191_gb300 as wdp

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    W = WORKLOAD
    dims, kappa, tol, delta = W["dims"], W["kappa"], W["tol"], W["delta"]
    inner = wdp.PREC_BY_NAME[args.inner]
    solver = wdp.BICGSTAB if args.solver == "bicgstab" else wdp.CGNR
    V = li.volume(dims)
    U = li.gauge(dims, W["eps"], W["gauge_seed"])
    b = li.gaussian_spinor(dims, W["source_seed"])
    wd = wdp.WilsonDirac(dims)
    wd.load_gauge(U)
    s = wd.stream
    fb = wd.upload(b, wdp.F64)
    fx = wd.new_field(wdp.F64, 2)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    def solve(prec):
        return wd.solve_device(fx, fb, kappa, tol=tol, delta=delta, solver=solver, inner_precision=prec)

    for _ in range(args.warmup):
        solve(inner)
    torch.cuda.synchronize()

    # ---- timed region: K whole solves, inputs resident in HBM
    times, launches, infos = [], 0, []
    with ClockSampler(local) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.add_(1)  # L2 flush between timed solves
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            r = solve(inner)
            e1.record(s)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1000.0)
            launches += r.kernel_launches
            infos.append(r)
        torch.cuda.synchronize()
        barrier(ws)
    clocks = clk.summary()
    t_total = max_over_ranks(ws, sum(times))
    value = ws * args.steps / t_total
    r0 = infos[-1]
    assert r0.status == 0 and r0.true_rel_residual <= tol, r0

    # ---- pure FP64 solve of the same system (the comparison of the metric)
    f64_times, f64_info = [], None
    for _ in range(max(1, args.fp64_solves)):
        flush.add_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        f64_info = solve(wdp.F64)
        e1.record(s)
        e1.synchronize()
        f64_times.append(e0.elapsed_time(e1) / 1000.0)
    f64_s = statistics.mean(f64_times)

    # ---- end to end through wd_solve with pinned host buffers
    bh = torch.from_numpy(b.view(np.float64).reshape(-1)).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    e2e_t = []
    for k in range(args.steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = wd.solve(xh, bh, kappa, tol=tol, delta=delta, solver=solver, inner_precision=inner)
        dt = time.perf_counter() - t0
        if k > 0:
            e2e_t.append(dt)
        assert r.status == 0
    e2e_value = ws * len(e2e_t) / max_over_ranks(ws, sum(e2e_t))

    # ---- roofline of the dominant kernel: the inner-precision dslash on this
    # lattice, same launch configuration as inside the solve, L2 flushed
    t_ds = time_dslash(wd, torch, inner, 50, flush=flush)
    vh = V // 2
    bytes_launch = BYTES_PER_SITE[inner] * vh
    hbm, src = peaks()
    achieved = bytes_launch / t_ds / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": None, "peak_source": src,
                "kernel": f"dslash {args.inner} 12-real, {dims[0]}^3x{dims[3]}, {vh} sites/launch, "
                          f"{BYTES_PER_SITE[inner]} B/site algorithmic", "us_per_launch": round(t_ds * 1e6, 2)}

    line = {"metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1000 * t_total / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.inner + "+f64", "data": "synthetic",
            "config": {"workload": W["workload"], "lattice": "24x24x24x64", "solver": args.solver,
                       "inner_precision": args.inner, "parallelism": f"replicas{ws}",
                       "l2": "flushed between timed solves (256 MB write); inputs (FP64 gauge 340 MB) exceed L2"},
            "solve": {"iters": r0.iters, "reliable_updates": r0.reliable_updates,
                      "true_rel_residual": r0.true_rel_residual},
            "fp64_solve": {"ms_per_solve": round(1000 * f64_s, 3), "iters": f64_info.iters,
                           "true_rel_residual": f64_info.true_rel_residual},
            "speedup_vs_fp64": round(f64_s / (t_total / args.steps), 3),
            "e2e": {"value": round(e2e_value, 4), "unit": "solves/s", "h2d_bytes_per_step": V * 24 * 8,
                    "d2h_bytes_per_step": V * 24 * 8},
            "gpu_launches": launches, "roofline": roofline, "clocks": clocks}

    # ---- dslash bandwidth sweep on the large lattice (inputs >> L2)
    if args.sweep and rank == 0:
        del wd
        torch.cuda.empty_cache()
        line["dslash_sweep"] = dslash_sweep(torch, args)

    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(U, b, dims, kappa, oracle_iterations(kappa), args.cpu_iters)
    if rank == 0:
        print(json.dumps(line))
    return 0


def dslash_sweep(torch, args):
    import lattice_inputs as li
    import paper_0911_3191_gb300 as wdp
    dims = tuple(int(x) for x in args.sweep_dims.split(","))
    V = li.volume(dims)
    t0 = time.perf_counter()
    U = li.gauge(dims, 0.3, 1002)
    gen_s = time.perf_counter() - t0
    wd = wdp.WilsonDirac(dims)
    wd.load_gauge(U)
    del U
    hbm, src = peaks()
    out = {"lattice": "x".join(map(str, dims)), "gauge_gen_s": round(gen_s, 1)}
    for prec in (0, 1, 2, 3, 4):
        t = time_dslash(wd, torch, prec, 20)
        gbs = BYTES_PER_SITE[prec] * (V // 2) / t / 1e9
        out[PREC_NAME[prec]] = {"us": round(t * 1e6, 1), "GB/s": round(gbs, 1), "frac": round(gbs / hbm, 4),
                                "eff_gflops": round(FLOPS_PER_SITE * (V // 2) / t / 1e9, 1)}
    out["peak_gbs"] = hbm
    out["peak_source"] = src
    wd.close()
    return out


def run_dslash_only(args):
    import torch

    import lattice_inputs as li
    import paper_0911_3191_gb300 as wdp
    dims = tuple(int(x) for x in args.sweep_dims.split(","))
    prec = wdp.PREC_BY_NAME[args.dslash_only]
    wd = wdp.WilsonDirac(dims)
    wd.load_gauge(li.gauge(dims, 0.3, 1002))
    fin = wd.new_field(prec)
    fin.zero_()
    fout = wd.new_field(prec)
    for _ in range(args.warmup + args.steps):
        wd.dslash(fout, fin, wdp.EVEN, False, prec)
    torch.cuda.synchronize()
    t = time_dslash(wd, torch, prec, max(1, args.steps))
    vh = li.volume(dims) // 2
    gbs = BYTES_PER_SITE[prec] * vh / t / 1e9
    print(json.dumps({"dslash": args.dslash_only, "lattice": "x".join(map(str, dims)), "us": round(t * 1e6, 2),
                      "GB/s": round(gbs, 1), "frac": round(gbs / peaks()[0], 4)}))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner", default="q16", choices=["f64", "f32", "q16", "h16n", "b16n"])
    ap.add_argument("--solver", default="bicgstab", choices=["bicgstab", "cgnr"])
    ap.add_argument("--fp64-solves", type=int, default=2)
    ap.add_argument("--no-sweep", dest="sweep", action="store_false")
    ap.add_argument("--sweep-dims", default="64,64,64,128")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=20)
    ap.add_argument("--dslash-only", default=None, choices=["f64", "f32", "q16", "h16n", "b16n"],
                    help="time only the dslash of one precision on --sweep-dims (profiling case)")
    args = ap.parse_args()
    if args.dslash_only:
        return run_dslash_only(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
