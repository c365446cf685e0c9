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


def bytes_per_site(prec, recon, tfix=False, recon8=False):
    """Compulsory bytes of one output site: the links read (8, or 6 in the
    temporal gauge, asymptotically: the last time slice still reads its
    temporal links), one input and one output spinor; FP64 links hold
    ``recon`` reals, FP32 / 16-bit links 12 reals or 8 numbers (recon8)."""
    if prec == 0:
        link = 8 * recon
    else:
        link = {1: 48, 2: 24, 3: 24, 4: 24}[prec] * (8 if recon8 else 12) // 12
    spinor = {0: 192, 1: 96, 2: 52, 3: 52, 4: 52}[prec]
    return (6 if tfix else 8) * link + 2 * spinor


def flops_per_site(tfix=False):
    """The paper's 1320 flops per site; the temporal gauge removes the two
    temporal SU(3) multiplies (2 x 132 flops) away from the last time slice."""
    return FLOPS_PER_SITE - (2 * 132 if tfix else 0)


FLOPS_PER_SITE = 1320  # the paper's effective count (Sec. 4.3)
# FP64 FMA peak of one GB300, measured with an FMA-throughput loop (1.252 TFLOP/s);
# the unit count agrees: 2 FP64 FMA lanes per SM per clock x 2 flops x 152 SMs
# x 2.07 GHz = 1.259 TFLOP/s
FP64_PEAK_TFLOPS = 1.252
# DRAM bytes of one launch (dram__bytes_read.sum + dram__bytes_write.sum)
# from an ncu capture of the dslash-only command of this file, keyed by
# (precision, link reals, lattice, temporal gauge).  KERNEL_SOURCES_SHA is the
# hash of the kernel sources the counters were taken on (kernel_sources_sha());
# when the sources differ, the bench reports traffic as null.
KERNEL_SOURCES_SHA = "b32b36328ca2fb9b"
NCU_TRAFFIC_BYTES = {("f64", 18, "24x24x24x64", True): 5.238e+08, ("q16", 12, "24x24x24x64", True): 8.946e+07}


def kernel_sources_sha() -> str:
    """sha256 (16 hex digits) of the CUDA sources that define the dslash kernels."""
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_0911_3191_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(csrc, "*.cuh")) + glob.glob(os.path.join(csrc, "wd_prec_*.cu"))):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(key):
    """The recorded DRAM traffic of a kernel, or None when the kernel sources
    changed since it was captured."""
    if not KERNEL_SOURCES_SHA or kernel_sources_sha() != KERNEL_SOURCES_SHA:
        return None
    return NCU_TRAFFIC_BYTES.get(key)
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
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_iterations(kappa: float) -> int:
    with open(ORACLE_ITERS) as f:
        d = json.load(f)
    return int(d["bicgstab_schur"][f"{kappa:.3f}"]["iterations"])


def cpu_baseline(U, b, dims, kappa, iters_full: int, sample_iters: int):
    """The oracle as it stands: FP64 BiCGstab on the Schur system, a bounded
    sample of iterations.  What ran is reported as it ran (sample_seconds for
    sample_iterations); the solves/s value extrapolates it to a full solve of
    iters_full iterations (scale = iters_full / sample_iterations)."""
    import oracle
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    oracle._load()
    t0 = time.perf_counter()
    oracle.bicgstab_schur_iterations(b, U, dims, kappa, sample_iters)
    dt = time.perf_counter() - t0
    per_solve = dt / sample_iters * iters_full
    return {"value": 1.0 / per_solve, "unit": "solves/s", "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle", "sample_iterations": sample_iters, "sample_seconds": round(dt, 6),
            "full_solve_iterations": iters_full, "scale": round(iters_full / sample_iters, 4),
            "extrapolated": True,
            "sample": f"{sample_iters} FP64 BiCGstab iterations of the {dims[0]}^3x{dims[3]} Schur solve "
                      f"({dt:.1f} s measured); value = that rate scaled to the {iters_full} iterations of "
                      f"the full FP64 solve"}


def bench_config(args, ws):
    """The workload both arms report (the reference arm runs it on the CPU oracle)."""
    return {"workload": WORKLOAD["workload"], "lattice": "24x24x24x64", "solver": args.solver,
            "fp64_link_reals": args.recon, "temporal_gauge": args.temporal_gauge,
            "low_precision_links": "8 numbers" if args.recon8 else "12 reals",
            "loop": "host" if args.host_loop else "cuda-graph",
            "inner_precision": args.inner, "parallelism": f"replicas{ws}",
            "l2": "flushed between timed solves and launches (256 MB write, then 256 MB read); inputs (FP64 gauge 340 MB) exceed L2"}


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
    # a step is a bounded sample of the solve: `sample` FP64 BiCGstab
    # iterations of the same Schur system; ms_per_step is the measured time of
    # that step, and value extrapolates it to whole solves per second
    sample = 6
    for _ in range(args.warmup):
        cpu_baseline(U, b, dims, kappa, iters_full, 2)
    vals = [cpu_baseline(U, b, dims, kappa, iters_full, sample) for _ in range(args.steps)]
    step_s = statistics.mean(x["sample_seconds"] for x in vals)
    v = sample / (step_s * iters_full)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000.0 * step_s, 3),
            "step": f"{sample} of the {iters_full} FP64 BiCGstab iterations of one solve (measured); value = "
                    f"solves/s extrapolated by the factor {iters_full / sample:.3f}",
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, ws),
            "cpu_baseline": {**vals[0], "value": v, "sample_seconds": round(step_s, 6),
                             "sample": f"{sample} FP64 BiCGstab iterations of the {dims[0]}^3x{dims[3]} Schur "
                                       f"solve per step ({step_s:.1f} s measured, the mean over {args.steps} "
                                       f"steps); value = that rate scaled to the {iters_full} iterations of the "
                                       f"full FP64 solve"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


class L2Flush:
    """Empties the L2 (129 MB) between timed launches: writes a 256 MB
    buffer, then reads another 256 MB one.  The read evicts the dirty lines of
    the write (their write-back happens here, not inside the next timed
    launch), so a timed launch starts with none of its inputs in L2 and pays
    only for its own traffic."""

    def __init__(self, torch):
        n = 256 * 1024 * 1024 // 4
        self.torch = torch
        self.w = torch.empty(n, dtype=torch.float32, device="cuda")
        self.r = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.out = torch.empty((), dtype=torch.float32, device="cuda")

    def __call__(self):
        self.w.add_(1)
        self.torch.sum(self.r, dim=0, out=self.out)


def time_dslash(wd, torch, prec, n, flush=None, psi=None):
    """Average device time of one dslash launch (CUDA events on the
    library's stream), optionally flushing L2 between launches.  The input
    is the host spinor ``psi`` (odd sites) when given, else zeros."""
    import paper_0911_3191_gb300 as wdp
    if psi is not None:
        fin = wd.upload(psi, prec, parity=wdp.ODD)
    else:
        fin = wd.new_field(prec)
        fin.zero_()
    fout = wd.new_field(prec)
    s = wd.stream
    for _ in range(3):
        wd.dslash(fout, fin, wdp.EVEN, False, prec)
    ts = []
    for _ in range(n):
        if flush is not None:
            flush()
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
    wd.load_gauge(U, recon=args.recon, temporal_gauge=args.temporal_gauge, recon8=args.recon8)
    s = wd.stream
    fb = wd.upload(b, wdp.F64)
    fx = wd.new_field(wdp.F64, 2)
    flush = L2Flush(torch)

    def solve(prec):
        return wd.solve_device(fx, fb, kappa, tol=tol, delta=delta, solver=solver, inner_precision=prec,
                               use_graph=not args.host_loop)

    for _ in range(args.warmup):
        solve(inner)
    torch.cuda.synchronize()

    # ---- timed region: K whole solves, inputs resident in HBM
    times, launches, infos = [], 0, []
    with ClockSampler(local) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush()  # L2 flush between timed solves
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
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        f64_info = solve(wdp.F64)
        e1.record(s)
        e1.synchronize()
        f64_times.append(e0.elapsed_time(e1) / 1000.0)
    f64_s = statistics.mean(f64_times)

    # ---- the same solve with every inner precision (one timed solve each)
    by_inner = {}
    variants = [("f32", wdp.F32, False), ("q16", wdp.Q16, False), ("h16n", wdp.H16N, False),
                ("b16n", wdp.B16N, False), ("q16_xhat_f32", wdp.Q16, True), ("b16n_xhat_f32", wdp.B16N, True)]
    for name, prec, xf in variants:
        def solve_v():
            return wd.solve_device(fx, fb, kappa, tol=tol, delta=delta, solver=solver, inner_precision=prec,
                                   use_graph=not args.host_loop, xhat_f32=xf)
        solve_v()
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        ri = solve_v()
        e1.record(s)
        e1.synchronize()
        by_inner[name] = {"ms": round(e0.elapsed_time(e1), 3), "iters": ri.iters, "updates": ri.reliable_updates,
                          "true_rel_residual": ri.true_rel_residual}

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
    # the host link alone: the same bytes copied each way between the same
    # pinned buffers and a device array, timed with CUDA events, so that the
    # end-to-end overhead splits into the copies and the library's own work
    dev = torch.empty(bh.numel(), dtype=bh.dtype, device="cuda")
    cs = torch.cuda.Stream()
    h2d_ms, d2h_ms = [], []
    with torch.cuda.stream(cs):
        for k in range(4):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(cs)
            dev.copy_(bh, non_blocking=True)
            ev[1].record(cs)
            xh.copy_(dev, non_blocking=True)
            ev[2].record(cs)
            ev[2].synchronize()
            if k > 0:
                h2d_ms.append(ev[0].elapsed_time(ev[1]))
                d2h_ms.append(ev[1].elapsed_time(ev[2]))
    del dev
    nbytes = bh.numel() * bh.element_size()
    host_link = {"h2d_GB_per_s": round(nbytes / statistics.mean(h2d_ms) / 1e6, 1),
                 "d2h_GB_per_s": round(nbytes / statistics.mean(d2h_ms) / 1e6, 1),
                 "copies_ms": round(statistics.mean(h2d_ms) + statistics.mean(d2h_ms), 3),
                 "e2e_minus_device_ms": round(1000.0 * ws / e2e_value - 1000.0 * t_total / args.steps, 3)}

    # ---- rooflines.  The dominant kernel of the step is the FP64 dslash of the
    # reliable updates (about 60% of the solve by the host-loop launch list),
    # bound by the FP64 pipe: achieved = 1320 flops/site x Vh / launch time.
    # The inner-precision dslash (the "dslash GB/s" of the metric) is bound by
    # HBM: achieved = algorithmic bytes/site x Vh / launch time.  Both timed with
    # CUDA events on the library's stream, same lattice and launch
    # configuration as inside the solve, L2 flushed between launches.
    vh = V // 2
    t64 = time_dslash(wd, torch, wdp.F64, 20, flush=flush, psi=b)
    tf = args.temporal_gauge
    f64_tflops = flops_per_site(tf) * vh / t64 / 1e12
    traffic = ncu_traffic(("f64", args.recon, "x".join(map(str, dims)), tf))
    roofline = {"bound": "alu", "achieved": round(f64_tflops, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": round(f64_tflops / FP64_PEAK_TFLOPS, 4), "traffic": traffic,
                "algorithmic_bytes": bytes_per_site(0, args.recon, tf) * vh, "peak_source": "measured FP64 FMA",
                "kernel_sources_sha": kernel_sources_sha(),
                "kernel": f"dslash f64 {args.recon}-real (reliable update){' temporal gauge' if tf else ''}, "
                          f"{dims[0]}^3x{dims[3]}, {vh} sites/launch, {flops_per_site(tf)} flops/site",
                "us_per_launch": round(t64 * 1e6, 2)}
    t_ds = time_dslash(wd, torch, inner, 50, flush=flush, psi=b)
    hbm, src = peaks()
    achieved = bytes_per_site(inner, 12, tf, args.recon8) * vh / t_ds / 1e9
    dslash_roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                       "frac": round(achieved / hbm, 4),
                       "traffic": ncu_traffic((args.inner, 8 if args.recon8 else 12, "x".join(map(str, dims)), tf)),
                       "peak_source": src,
                       "kernel": f"dslash {args.inner} {'8-number' if args.recon8 else '12-real'} (inner iteration), "
                                 f"{dims[0]}^3x{dims[3]}, {vh} "
                                 f"sites/launch, {bytes_per_site(inner, 12, tf, args.recon8)} B/site algorithmic"
                                 f"{' (temporal gauge)' if tf else ''}",
                       "us_per_launch": round(t_ds * 1e6, 2)}

    line = {"metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1000 * t_total / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.inner + "+f64", "data": "synthetic",
            "config": bench_config(args, ws),
            "solve": {"iters": r0.iters, "reliable_updates": r0.reliable_updates,
                      "true_rel_residual": r0.true_rel_residual},
            "fp64_solve": {"ms_per_solve": round(1000 * f64_s, 3), "iters": f64_info.iters,
                           "true_rel_residual": f64_info.true_rel_residual},
            "speedup_vs_fp64": round(f64_s / (t_total / args.steps), 3),
            "solve_by_inner_precision": by_inner,
            "e2e": {"value": round(e2e_value, 4), "unit": "solves/s", "h2d_bytes_per_step": V * 24 * 8,
                    "d2h_bytes_per_step": V * 24 * 8, "host_link": host_link},
            "gpu_launches": launches, "roofline": roofline, "dslash_roofline": dslash_roofline, "clocks": clocks}

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
    psi = li.gaussian_spinor(dims, 2102)
    hbm, src = peaks()
    out = {"lattice": "x".join(map(str, dims)), "gauge_gen_s": round(gen_s, 1), "fp64_link_reals": args.recon,
           "input": "Gaussian spinor", "peak_gbs": hbm, "peak_source": src}
    # link storage variants: general links; temporal gauge; temporal gauge
    # with the 8-number FP32 / 16-bit links (the paper's "8 GF")
    for tf, r8 in ((False, False), (True, False), (True, True)):
        wd = wdp.WilsonDirac(dims)
        wd.load_gauge(U, recon=args.recon, temporal_gauge=tf, recon8=r8)
        for prec in (0, 1, 2, 3, 4):
            if r8 and prec == 0:
                continue
            t = time_dslash(wd, torch, prec, 20, psi=psi)
            nbytes = bytes_per_site(prec, args.recon, tf, r8)
            gbs = nbytes * (V // 2) / t / 1e9
            out[PREC_NAME[prec] + ("_temporal_gauge" if tf else "") + ("_recon8" if r8 else "")] = {
                "us": round(t * 1e6, 1), "GB/s": round(gbs, 1), "frac": round(gbs / hbm, 4), "bytes_per_site": nbytes,
                "eff_gflops": round(flops_per_site(tf) * (V // 2) / t / 1e9, 1)}
        wd.close()
    return out


def run_table(args):
    """The solver comparison on the 24^3x64 lattice (links exp(0.3 i H)):
    kappa in {0.12, 0.124} x 3 Gaussian sources x {BiCGstab, CGNR} x
    {pure FP64; reliable updates (Alg. 2, delta 0.1) with F32, Q16, H16N, B16N
    inner; defect correction (Alg. 1) with Q16 inner at eps_in 1e-1, 1e-2 and
    F32 inner at eps_in 1e-3 .. 1e-6}, all to |r|/|b| <= 1e-12.  Each entry:
    device time of one solve (inputs resident, L2 flushed), iterations
    (reliable updates / corrections included), FP64 updates, true residual."""
    import torch

    import lattice_inputs as li
    import paper_0911_3191_gb300 as wdp
    dims = WORKLOAD["dims"]
    U = li.gauge(dims, WORKLOAD["eps"], WORKLOAD["gauge_seed"])
    wd = wdp.WilsonDirac(dims)
    wd.load_gauge(U, recon=args.recon, temporal_gauge=args.temporal_gauge)
    del U
    flush = L2Flush(torch)
    fx = wd.new_field(wdp.F64, 2)
    variants = [("fp64", wdp.F64, 0.1, False)]
    variants += [(f"ru-{n}", p, 0.1, False) for n, p in (("f32", wdp.F32), ("q16", wdp.Q16), ("h16n", wdp.H16N),
                                                         ("b16n", wdp.B16N))]
    variants += [(f"dc-q16-{e:g}", wdp.Q16, e, True) for e in (1e-1, 1e-2)]
    variants += [(f"dc-f32-{e:g}", wdp.F32, e, True) for e in (1e-3, 1e-4, 1e-5, 1e-6)]
    rows = []
    for kappa in (0.12, 0.124):
        for seed in (2001, 2011, 2021):
            fb = wd.upload(li.gaussian_spinor(dims, seed), wdp.F64)
            for solver_name, solver in (("bicgstab", wdp.BICGSTAB), ("cgnr", wdp.CGNR)):
                for name, prec, delta, restart in variants:
                    def go():
                        return wd.solve_device(fx, fb, kappa, tol=1e-12, delta=delta, max_iter=4000,
                                               solver=solver, inner_precision=prec, restart=restart, check=False)
                    go()  # graph capture and tuning outside the timing
                    flush()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(wd.stream)
                    r = go()
                    e1.record(wd.stream)
                    e1.synchronize()
                    rows.append({"kappa": kappa, "source_seed": seed, "solver": solver_name, "variant": name,
                                 "ms": round(e0.elapsed_time(e1), 3), "iters": r.iters,
                                 "updates": r.reliable_updates, "true_rel_residual": r.true_rel_residual,
                                 "status": r.status})
            del fb
    wd.close()
    print(json.dumps({"table": "24x24x24x64 eps=0.3 solver comparison, tol 1e-12",
                      "temporal_gauge": args.temporal_gauge, "rows": rows}))
    return 0


def run_oracle_timing(args):
    """The FP64 CPU oracle timed on this host's cores, all of them and one:
    the dslash on 24^3x64 (and 64^3x128 with all cores) and full Schur
    BiCGstab solves on 8^3x16 (tol 1e-12) and, by a bounded sample of
    iterations scaled to the full iteration count, on 24^3x64."""
    out = {"host_cores": os.cpu_count(), "runs": {}}
    for threads in (os.cpu_count(), 1):
        env = dict(os.environ, OMP_NUM_THREADS=str(threads))
        cmd = [sys.executable, os.path.abspath(__file__), "--oracle-timing-child", str(threads)]
        r = subprocess.run(cmd, env=env, capture_output=True, text=True, check=True)
        out["runs"][str(threads)] = json.loads(r.stdout.strip().splitlines()[-1])
    print(json.dumps(out))
    return 0


def run_oracle_timing_child(threads):
    import oracle
    import lattice_inputs as li
    res = {"threads": threads}
    dims = (8, 8, 8, 16)
    U, b = li.gauge(dims, 0.5, 1000), li.gaussian_spinor(dims, 2000)
    t0 = time.perf_counter()
    _, st, iters, rel = oracle.solve(b, U, dims, 0.12, tol=1e-12)
    res["solve_8x8x8x16"] = {"s": round(time.perf_counter() - t0, 3), "iters": iters, "true_rel_residual": rel}
    dims = WORKLOAD["dims"]
    U, b = li.gauge(dims, WORKLOAD["eps"], WORKLOAD["gauge_seed"]), li.gaussian_spinor(dims, WORKLOAD["source_seed"])
    t0 = time.perf_counter()
    oracle.dslash(b, U, dims, out_parity=0)
    t = time.perf_counter() - t0
    vh = li.volume(dims) // 2
    res["dslash_24x24x24x64"] = {"s": round(t, 3), "ns_per_site": round(1e9 * t / vh, 1),
                                 "gflops": round(1320 * vh / t / 1e9, 2)}
    n = 10 if threads > 1 else 2
    t0 = time.perf_counter()
    oracle.bicgstab_schur_iterations(b, U, dims, WORKLOAD["kappa"], n)
    s_it = (time.perf_counter() - t0) / n
    full = oracle_iterations(WORKLOAD["kappa"])
    res["solve_24x24x24x64"] = {"s_per_iteration": round(s_it, 3), "iterations": full,
                                "s_est": round(s_it * full, 2), "sample_iterations": n}
    if threads > 1:
        del U, b
        dims = (64, 64, 64, 128)
        U, b = li.gauge(dims, 0.3, 1002), li.gaussian_spinor(dims, 2102)
        t0 = time.perf_counter()
        oracle.dslash(b, U, dims, out_parity=0)
        t = time.perf_counter() - t0
        vh = li.volume(dims) // 2
        res["dslash_" + "x".join(map(str, dims))] = {"s": round(t, 3), "ns_per_site": round(1e9 * t / vh, 1),
                                                     "gflops": round(1320 * vh / t / 1e9, 2)}
    print(json.dumps(res))
    return 0


def run_dslash_only(args):
    import torch

    import lattice_inputs as li
    import paper_0911_3191_gb300 as wdp
    dims = tuple(int(x) for x in args.sweep_dims.split(","))
    prec = wdp.PREC_BY_NAME[args.dslash_only]
    wd = wdp.WilsonDirac(dims)
    wd.load_gauge(li.gauge(dims, 0.3, 1002), recon=args.recon, temporal_gauge=args.temporal_gauge,
                  recon8=args.recon8)
    fin = wd.upload(li.gaussian_spinor(dims, 2102), prec, parity=wdp.ODD)
    fout = wd.new_field(prec)
    for _ in range(args.warmup + args.steps):
        wd.dslash(fout, fin, wdp.EVEN, False, prec)
    torch.cuda.synchronize()
    ts = []
    for _ in range(max(1, args.steps)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(wd.stream)
        wd.dslash(fout, fin, wdp.EVEN, False, prec)
        e1.record(wd.stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1000.0)
    t = statistics.mean(ts)
    vh = li.volume(dims) // 2
    gbs = bytes_per_site(prec, args.recon, args.temporal_gauge, args.recon8) * vh / t / 1e9
    print(json.dumps({"dslash": args.dslash_only, "lattice": "x".join(map(str, dims)),
                      "temporal_gauge": args.temporal_gauge, "recon8": args.recon8, "us": round(t * 1e6, 2),
                      "GB/s": round(gbs, 1), "frac": round(gbs / peaks()[0], 4)}))
    return 0


def run_slab(args):
    """T-slab decomposition (Sec. 6): one dslash of a lattice split into
    WORLD_SIZE slabs along T (one per rank; world 1 on one GPU exchanges with
    itself), through tslab.SlabDslash: face pack, face exchange on a second
    stream overlapping the interior slices, boundary slices.  Timed against
    the whole-lattice dslash kernel on the same rank's slab, general links,
    inputs beyond L2, CUDA events on the library's stream, max over ranks."""
    import numpy as np
    import torch

    import lattice_inputs as li
    import paper_0911_3191_gb300 as wdp
    from paper_0911_3191_gb300 import tslab
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dims = tuple(int(x) for x in args.sweep_dims.split(","))
    X, Y, Z, T = dims
    t0, nt = tslab.slab_range(T, ws, rank)
    ss = X * Y * Z
    slab = (X, Y, Z, nt)
    U = li.gauge(slab, 0.3, 1002 + rank)  # each rank its own slab of links (synthetic)
    psi = li.gaussian_spinor(slab, 2102 + rank)
    wd = wdp.WilsonDirac(slab)
    wd.load_gauge(U, recon=args.recon)
    del U
    sd = tslab.SlabDslash(wd, rank, ws, t_antiperiodic=True)
    out = {"lattice": "x".join(map(str, dims)), "ranks": ws, "slab": "x".join(map(str, slab)),
           "links": "general (no temporal gauge)", "fp64_link_reals": args.recon}
    vh = li.volume(slab) // 2
    hbm, src = peaks()
    for name in ("f64", "f32", "q16", "h16n", "b16n"):
        prec = wdp.PREC_BY_NAME[name]
        fin = wd.upload(psi, prec, parity=wdp.ODD)
        fout = wd.new_field(prec)

        def timed(fn, n):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            barrier(ws)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(wd.stream)
            for _ in range(n):
                fn()
            e1.record(wd.stream)
            e1.synchronize()
            return max_over_ranks(ws, e0.elapsed_time(e1) / 1000.0 / n)

        n = max(5, args.steps)
        t_slab = timed(lambda: sd.apply(fout, fin, wdp.EVEN, False, prec), n)
        t_whole = timed(lambda: wd.dslash(fout, fin, wdp.EVEN, False, prec), n)
        face = wd.slab_face_bytes(prec)
        nbytes = bytes_per_site(prec, args.recon) * vh
        out[name] = {"slab_us": round(t_slab * 1e6, 1), "whole_kernel_us": round(t_whole * 1e6, 1),
                     "overhead": round(t_slab / t_whole - 1.0, 4),
                     "slab_GB/s_per_rank": round(nbytes / t_slab / 1e9, 1),
                     "slab_frac_of_hbm": round(nbytes / t_slab / 1e9 / hbm, 4),
                     "face_bytes_exchanged_per_dslash": 2 * face}
        del fin, fout
    out["peak_gbs"], out["peak_source"] = hbm, src
    if rank == 0:
        print(json.dumps({"slab_dslash": out}))
    return 0


def run_large_solve(args):
    """The large-lattice solve: 64^3 x 128 (33.5M sites), links exp(0.3 i H),
    12-real FP64 links, kappa 0.124, Gaussian source; CG on the normal
    equations to |b - M x| / |b| <= 1e-10, mixed (Q16 inner iteration, FP64
    reliable updates, delta 0.1) against pure FP64 on the same lattice
    (Sec. 5.4: time to solution).  Inputs resident in HBM, CUDA events on the
    library's stream; each returned x is checked by the CPU oracle's M on the
    whole lattice."""
    import numpy as np
    import torch

    import lattice_inputs as li
    import oracle
    import paper_0911_3191_gb300 as wdp
    dims = tuple(int(x) for x in args.sweep_dims.split(","))
    kappa, tol = 0.124, 1e-10
    t0 = time.perf_counter()
    U = li.gauge(dims, 0.3, 1002)
    b = li.gaussian_spinor(dims, 2103)
    gen_s = time.perf_counter() - t0
    wd = wdp.WilsonDirac(dims)
    wd.load_gauge(U, recon=12, temporal_gauge=args.temporal_gauge)
    fb = wd.upload(b, wdp.F64)
    fx = wd.new_field(wdp.F64, 2)
    out = {"lattice": "x".join(map(str, dims)), "kappa": kappa, "tol": tol, "solver": "cgnr",
           "fp64_link_reals": 12, "temporal_gauge": args.temporal_gauge, "gauge_gen_s": round(gen_s, 1)}
    with ClockSampler(0) as clk:
        for name, prec in (("mixed_q16", wdp.Q16), ("fp64", wdp.F64)):
            if prec == wdp.Q16:  # warm-up (graph build, gauge copy)
                wd.solve_device(fx, fb, kappa, tol=tol, delta=0.1, solver=wdp.CGNR, inner_precision=prec)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(wd.stream)
            r = wd.solve_device(fx, fb, kappa, tol=tol, delta=0.1, solver=wdp.CGNR, inner_precision=prec)
            e1.record(wd.stream)
            e1.synchronize()
            x = wd.download(fx, wdp.F64)
            t1 = time.perf_counter()
            rel = oracle.true_residual(x, b, U, dims, kappa)
            out[name] = {"s": round(e0.elapsed_time(e1) / 1000.0, 4), "iters": r.iters,
                         "reliable_updates": r.reliable_updates, "status": r.status,
                         "true_rel_residual": r.true_rel_residual, "oracle_true_rel_residual": rel,
                         "oracle_check_s": round(time.perf_counter() - t1, 1)}
            assert r.status == 0 and rel <= tol, (name, r, rel)
    out["speedup_mixed_vs_fp64"] = round(out["fp64"]["s"] / out["mixed_q16"]["s"], 3)
    out["clocks"] = clk.summary()
    out["oracle_cores"] = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    print(json.dumps({"large_solve": out}))
    return 0


def run_multishift(args):
    """Multi-shift solves (wd_solve_multishift_device) on the batched workload:
    32^3 x 64 lattice (links exp(0.3 i H)), the 12 spin-colour point sources at
    the origin, each solved for kappa in {0.118, 0.12, 0.122, 0.124} by one
    shared FP32 multi-shift iteration plus a reliable-update refinement per
    kappa (Q16 inner) to 1e-12; plus one Gaussian source (two shifted
    families).  Timed against the same systems solved one at a time."""
    import numpy as np
    import torch

    import lattice_inputs as li
    import paper_0911_3191_gb300 as wdp
    dims = (32, 32, 32, 64)
    kappas = [0.118, 0.12, 0.122, 0.124]
    inner = wdp.PREC_BY_NAME[args.inner]
    wd = wdp.WilsonDirac(dims)
    wd.load_gauge(li.gauge(dims, 0.3, 1003), recon=args.recon, temporal_gauge=args.temporal_gauge)
    V = li.volume(dims)
    full = 2 * wd.field_bytes(wdp.F64)
    s = wd.stream
    host = np.zeros((V, 4, 3), dtype=np.complex128)
    srcs = []
    for sp in range(4):
        for co in range(3):
            host[0, sp, co] = 1.0
            srcs.append(("point", wd.upload(host, wdp.F64)))
            host[0, sp, co] = 0.0
    srcs.append(("gaussian", wd.upload(li.gaussian_spinor(dims, 2600), wdp.F64)))
    fx = wd.new_field(wdp.F64, 2 * len(kappas))
    fx1 = wd.new_field(wdp.F64, 2)

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        out = fn()
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1000.0, out

    wd.solve_multishift_device(fx, srcs[0][1], kappas, tol=1e-12, inner_precision=inner)  # warm-up
    wd.solve_device(fx1, srcs[0][1], kappas[0], tol=1e-12, inner_precision=inner)
    rows = {"point": [0.0, 0.0, 0], "gaussian": [0.0, 0.0, 0]}
    iters, worst = [], 0.0
    with ClockSampler(0) as clk:
        for kind, fb in srcs:
            t_ms, infos = timed(lambda: wd.solve_multishift_device(fx, fb, kappas, tol=1e-12, inner_precision=inner))
            assert all(i.status == 0 and i.true_rel_residual <= 1e-12 for i in infos), infos
            worst = max(worst, max(i.true_rel_residual for i in infos))
            iters.append([i.iters for i in infos])
            t_solo = 0.0
            for k in kappas:
                t1, r1 = timed(lambda: wd.solve_device(fx1, fb, k, tol=1e-12, inner_precision=inner))
                assert r1.status == 0
                t_solo += t1
            rows[kind][0] += t_ms
            rows[kind][1] += t_solo
            rows[kind][2] += 1
    out = {"multishift": "32x32x32x64, 12 point sources + 1 Gaussian source, kappa " + ",".join(map(str, kappas)),
           "inner": args.inner, "temporal_gauge": args.temporal_gauge, "tol": 1e-12,
           "stage": "FP32 multi-shift BiCGstab to 1e-7, then reliable-update refinement per kappa",
           "max_true_rel_residual": worst, "iters_per_kappa_first_sources": iters[:2] + iters[-1:],
           "clocks": clk.summary()}
    for kind, (tm, ts, cnt) in rows.items():
        out[kind] = {"sources": cnt, "multishift_s": round(tm, 4), "one_at_a_time_s": round(ts, 4),
                     "speedup": round(ts / tm, 3) if tm else None}
    print(json.dumps(out))
    return 0


def run_batch(args):
    """Batched multi-RHS solve: 12 point-source spin-colour right-hand sides x
    4 kappa = 48 systems on a 32^3 x 64 lattice (links exp(0.3 i H)), Q16 inner
    BiCGstab with FP64 reliable updates to 1e-12, in one batched graph; timed
    against the same systems solved one at a time."""
    import numpy as np
    import torch

    import lattice_inputs as li
    import paper_0911_3191_gb300 as wdp
    dims = (32, 32, 32, 64)
    kappas = [0.118, 0.12, 0.122, 0.124]
    inner = wdp.PREC_BY_NAME[args.inner]
    wd = wdp.WilsonDirac(dims)
    wd.load_gauge(li.gauge(dims, 0.3, 1003), recon=args.recon, temporal_gauge=args.temporal_gauge)
    V = li.volume(dims)
    pts = [(s, c) for s in range(4) for c in range(3)]
    n = len(pts) * len(kappas)
    full = 2 * wd.field_bytes(wdp.F64)
    fb = wd.new_field(wdp.F64, 2 * n)
    host = np.zeros((V, 4, 3), dtype=np.complex128)
    ks = []
    r = 0
    for k in kappas:
        for (sp, co) in pts:
            host[0, sp, co] = 1.0
            f = fb[r * full:(r + 1) * full]
            wd.field_import(f[:full // 2], host, wdp.EVEN, wdp.F64)
            wd.field_import(f[full // 2:], host, wdp.ODD, wdp.F64)
            host[0, sp, co] = 0.0
            ks.append(k)
            r += 1
    fx = wd.new_field(wdp.F64, 2 * n)
    s = wd.stream
    # the autotuner writes its choice (RHS tile, grid, packed layout) to this cache
    tune_file = tempfile.NamedTemporaryFile(prefix="wd_tune_", suffix=".txt", delete=False).name
    os.environ["WD_TUNE_CACHE"] = tune_file
    t0 = time.perf_counter()
    infos = wd.solve_batch_device(fx, fb, ks, tol=1e-12, inner_precision=inner)  # includes the autotuning
    first_s = time.perf_counter() - t0
    for _ in range(max(0, args.warmup - 1)):
        wd.solve_batch_device(fx, fb, ks, tol=1e-12, inner_precision=inner)
    times = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            infos = wd.solve_batch_device(fx, fb, ks, tol=1e-12, inner_precision=inner)
            e1.record(s)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1000.0)
    assert all(i.status == 0 and i.true_rel_residual <= 1e-12 for i in infos), infos
    t_batch = statistics.mean(times)
    # the same systems one at a time (a sample of 8, scaled to 48)
    sample = list(range(0, n, n // 8))
    t_single = 0.0
    fx1 = wd.new_field(wdp.F64, 2)
    for q in sample:
        wd.solve_device(fx1, fb[q * full:(q + 1) * full], ks[q], tol=1e-12, inner_precision=inner)  # warm
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        r1 = wd.solve_device(fx1, fb[q * full:(q + 1) * full], ks[q], tol=1e-12, inner_precision=inner)
        e1.record(s)
        e1.synchronize()
        assert r1.status == 0
        t_single += e0.elapsed_time(e1) / 1000.0
    t_single *= n / len(sample)
    # the multi-RHS dslash against n single-RHS launches, inner precision
    del fx, fx1
    fin = wd.new_field(inner, n)
    fin.zero_()
    fout = wd.new_field(inner, n)
    fbi = wd.field_bytes(inner)
    ds = {}
    for label in ("batched", "single"):
        for rep in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            if label == "batched":
                wd.dslash_batch(fout, fin, n, wdp.EVEN, False, inner)
            else:
                for q in range(n):
                    wd.dslash(fout[q * fbi:(q + 1) * fbi], fin[q * fbi:(q + 1) * fbi], wdp.EVEN, False, inner)
            e1.record(s)
            e1.synchronize()
            if rep:
                ds.setdefault(label, []).append(e0.elapsed_time(e1) / 1000.0)
    vh = li.volume(dims) // 2
    t_b, t_s = statistics.mean(ds["batched"]), statistics.mean(ds["single"])
    mrhs = {"batched_us": round(1e6 * t_b, 1), "single_x_n_us": round(1e6 * t_s, 1),
            "batched_GB_per_s_algorithmic": round((8 * 24 + 2 * 52 * n) * vh / t_b / 1e9, 1)}
    # the FP64 (reliable-update) dslash, batched against single launches
    del fin, fout
    n64 = 16
    f64in = wd.new_field(wdp.F64, n64)
    f64in.zero_()
    f64out = wd.new_field(wdp.F64, n64)
    fb64 = wd.field_bytes(wdp.F64)
    d64 = {}
    for label in ("batched", "single"):
        for rep in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            if label == "batched":
                wd.dslash_batch(f64out, f64in, n64, wdp.EVEN, False, wdp.F64)
            else:
                for q in range(n64):
                    wd.dslash(f64out[q * fb64:(q + 1) * fb64], f64in[q * fb64:(q + 1) * fb64], wdp.EVEN, False,
                              wdp.F64)
            e1.record(s)
            e1.synchronize()
            if rep:
                d64.setdefault(label, []).append(e0.elapsed_time(e1) / 1000.0)
    mrhs["f64_batched16_us"] = round(1e6 * statistics.mean(d64["batched"]), 1)
    mrhs["f64_single_x16_us"] = round(1e6 * statistics.mean(d64["single"]), 1)
    del f64in, f64out
    try:
        shape = open(tune_file).read().strip().split("|")[-1].split()
        tuned = {"rhs_tile": int(shape[0]), "grid": int(shape[1]), "packed_pairs": bool(int(shape[2]))}
    except Exception:
        tuned = None
    os.unlink(tune_file)
    print(json.dumps({"batch": "32x32x32x64, 12 point sources x 4 kappa", "n_systems": n, "inner": args.inner,
                      "temporal_gauge": args.temporal_gauge, "tuned_shape": tuned,
                      "mrhs_dslash": mrhs,
                      "fp64_link_reals": args.recon, "s_per_batched_solve": round(t_batch, 4),
                      "systems_per_s": round(n / t_batch, 3), "s_first_call_incl_tuning": round(first_s, 3),
                      "s_one_at_a_time_est": round(t_single, 4), "batch_speedup": round(t_single / t_batch, 3),
                      "iters": [i.iters for i in infos], "reliable_updates": [i.reliable_updates for i in infos],
                      "max_true_rel_residual": max(i.true_rel_residual for i in infos), "clocks": clk.summary()}))
    return 0


def run_serve(args):
    """Serving stream: Poisson arrivals (exponential gaps, seed 3000) at 200/s
    of solve requests on 8 resident gauge fields (2 per volume: 16^3x32,
    24^3x48, 32^3x64, 48^3x96; links exp(0.3 i H)), kappa ~ U[0.115, 0.124],
    tol in {1e-8, 1e-10, 1e-12}, device-memory budget 80 GB, continuous
    batching through wd_server_*.  Each volume's requests share one Gaussian
    source and one host solution buffer (the client does not keep every
    solution); every request's FP64 true residual is reported by the server."""
    import numpy as np
    import torch

    import lattice_inputs as li
    import paper_0911_3191_gb300 as wdp
    vols = [(16, 16, 16, 32), (24, 24, 24, 48), (32, 32, 32, 64), (48, 48, 48, 96)]
    rng = np.random.default_rng(3000)
    n = args.serve_requests
    gaps = rng.exponential(1.0 / 200.0, size=n)
    arrival = np.cumsum(gaps) - gaps[0]
    vol_idx = rng.integers(0, 4, size=n)
    allowed = [int(v) for v in args.serve_volumes.split(",")]
    vol_idx = np.array([allowed[int(v) % len(allowed)] for v in vol_idx])
    field_idx = rng.integers(0, 2, size=n)
    kappas = rng.uniform(0.115, 0.124, size=n)
    tols = np.array([1e-8, 1e-10, 1e-12])[rng.integers(0, 3, size=n)]
    inner = wdp.PREC_BY_NAME[args.inner]
    srv = wdp.Server(budget_bytes=80 * 1000**3, max_slots=args.serve_slots, iters_per_step=args.serve_iters,
                     inner_precision=inner, delta=0.1, temporal_gauge=args.temporal_gauge, rhs_tile=args.serve_tile)
    gids, srcs, outs = {}, {}, {}
    t0 = time.perf_counter()
    for v, dims in enumerate(vols):
        for f in range(2):
            gids[(v, f)] = srv.add_gauge(dims, li.gauge(dims, 0.3, 1100 + 2 * v + f), recon=args.recon)
        # the client keeps its fields in page-locked host memory (as the
        # end-to-end solve of the benchmark does), so the server's transfers
        # run as DMA from pinned pages it does not have to register
        src = li.gaussian_spinor(dims, 2400 + v)
        srcs[v] = torch.empty(src.shape, dtype=torch.complex128).pin_memory().numpy()
        srcs[v][...] = src
        outs[v] = torch.zeros(src.shape, dtype=torch.complex128).pin_memory().numpy()
        del src
    setup_s = time.perf_counter() - t0
    pending, lat, infos = {}, [], []
    t_step = t_poll = 0.0
    nxt = 0
    start = time.perf_counter()
    with ClockSampler(0) as clk:
        while nxt < n or pending:
            now = time.perf_counter() - start
            while nxt < n and arrival[nxt] <= now:
                v = int(vol_idx[nxt])
                rid = srv.submit(gids[(v, int(field_idx[nxt]))], srcs[v], float(kappas[nxt]), float(tols[nxt]),
                                 x=outs[v])
                pending[rid] = (nxt, float(tols[nxt]))
                nxt += 1
            if not pending:
                time.sleep(max(0.0, min(arrival[nxt] - now, 0.01)))
                continue
            t_a = time.perf_counter()
            srv.step()
            tnow = time.perf_counter() - start
            t_step += time.perf_counter() - t_a
            t_a = time.perf_counter()
            for rid in list(pending):
                f, res, _ = srv.poll(rid)
                if f:
                    i, tol = pending.pop(rid)
                    lat.append(tnow - arrival[i])
                    infos.append((res, tol, int(vol_idx[i])))
            t_poll += time.perf_counter() - t_a
    makespan = time.perf_counter() - start
    server_stats = srv.stats()
    srv.close()
    # the same work done one solve at a time, inputs resident: one timed solo
    # solve per (volume, tol) at the middle kappa 0.1195, summed over the requests
    import torch
    solo = {}
    for v, dims in enumerate(vols):
        wd = wdp.WilsonDirac(dims)
        wd.load_gauge(li.gauge(dims, 0.3, 1100 + 2 * v), recon=args.recon, temporal_gauge=args.temporal_gauge)
        fb = wd.upload(srcs[v], wdp.F64)
        fx = wd.new_field(wdp.F64, 2)
        for tol in (1e-8, 1e-10, 1e-12):
            wd.solve_device(fx, fb, 0.1195, tol=tol, inner_precision=inner)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            wd.solve_device(fx, fb, 0.1195, tol=tol, inner_precision=inner)
            torch.cuda.synchronize()
            solo[(v, tol)] = time.perf_counter() - t1
        wd.close()
    serial = sum(solo[(int(vol_idx[i]), float(tols[i]))] for i in range(n))
    ok = sum(1 for r, tol, _ in infos if r.status == 0 and r.true_rel_residual <= tol)
    failures = [{"status": r.status, "true_rel_residual": r.true_rel_residual, "tol": tol, "iters": r.iters,
                 "volume": "x".join(map(str, vols[v]))}
                for r, tol, v in infos if not (r.status == 0 and r.true_rel_residual <= tol)]
    lat_a = np.array(lat)
    per_vol = {}
    for v, dims in enumerate(vols):
        lv = np.array([lat[k] for k in range(len(lat)) if infos[k][2] == v])
        if len(lv):
            per_vol["x".join(map(str, dims))] = {"n": int(len(lv)), "p50_s": round(float(np.percentile(lv, 50)), 3),
                                                 "p99_s": round(float(np.percentile(lv, 99)), 3)}
    print(json.dumps({"serve": f"{n} Poisson requests at 200/s, 4 volumes, 8 resident gauge fields, budget 80 GB",
                      "temporal_gauge": args.temporal_gauge,
                      "inner": args.inner, "requests": n, "converged_to_tol": ok, "makespan_s": round(makespan, 3),
                      "solves_per_s": round(n / makespan, 3),
                      "latency_p50_s": round(float(np.percentile(lat_a, 50)), 3),
                      "latency_p99_s": round(float(np.percentile(lat_a, 99)), 3), "per_volume": per_vol,
                      "setup_s": round(setup_s, 1), "max_slots": args.serve_slots, "iters_per_step": args.serve_iters,
                      "rhs_tile": args.serve_tile,
                      "one_at_a_time_s": round(serial, 2), "efficiency_vs_one_at_a_time": round(serial / makespan, 3),
                      "server_stats": server_stats, "host_step_s": round(t_step, 2), "host_poll_s": round(t_poll, 2),
                      "failures": failures[:10],
                      "solo_s": {f"{'x'.join(map(str, vols[v]))} tol {t:g}": round(x, 4) for (v, t), x in solo.items()},
                      "clocks": clk.summary()}))
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
    ap.add_argument("--temporal-gauge", action=argparse.BooleanOptionalAction, default=True,
                    help="load the links in the temporal gauge (Sec. 4.3; default on)")
    ap.add_argument("--recon8", action=argparse.BooleanOptionalAction, default=False,
                    help="FP32 / 16-bit links as the 8 numbers of App. A.2")
    ap.add_argument("--recon", type=int, default=18, choices=[12, 18],
                    help="reals stored per FP64 link (lower precisions always store 12)")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the solver loop from the host (profiling: ncu lists every kernel)")
    ap.add_argument("--cpu-iters", type=int, default=20)
    ap.add_argument("--dslash-only", default=None, choices=["f64", "f32", "q16", "h16n", "b16n"],
                    help="time only the dslash of one precision on --sweep-dims (profiling case)")
    ap.add_argument("--batch", action="store_true", help="batched 48-system multi-RHS solve (32^3x64)")
    ap.add_argument("--multishift", action="store_true", help="multi-shift solves over 4 kappa (32^3x64)")
    ap.add_argument("--serve", action="store_true", help="continuous-batching serving stream")
    ap.add_argument("--large-solve", action="store_true",
                    help="mixed vs FP64 CGNR to 1e-10 on --sweep-dims (64^3x128), oracle-checked")
    ap.add_argument("--slab", action="store_true",
                    help="T-slab decomposed dslash (one slab per rank, face exchange) on --sweep-dims")
    ap.add_argument("--oracle-timing", action="store_true",
                    help="time the FP64 CPU oracle (dslash, solves) on all host cores and on one")
    ap.add_argument("--oracle-timing-child", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--table", action="store_true",
                    help="solver comparison table on 24^3x64 (reliable update vs defect correction vs FP64)")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-iters", type=int, default=8)
    ap.add_argument("--serve-tile", type=int, default=0, choices=[-1, 0, 1, 2, 4],
                    help="systems per link tile of the inner dslash (-1 one per block row, 0 automatic)")
    ap.add_argument("--serve-volumes", default="0,1,2,3",
                    help="which of the four volumes (16^3x32, 24^3x48, 32^3x64, 48^3x96) requests go to")
    args = ap.parse_args()
    if args.batch:
        return run_batch(args)
    if args.serve:
        return run_serve(args)
    if args.multishift:
        return run_multishift(args)
    if args.slab:
        return run_slab(args)
    if args.large_solve:
        return run_large_solve(args)
    if args.table:
        return run_table(args)
    if args.oracle_timing_child:
        return run_oracle_timing_child(args.oracle_timing_child)
    if args.oracle_timing:
        return run_oracle_timing(args)
    if args.dslash_only:
        return run_dslash_only(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
