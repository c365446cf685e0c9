"""bench.py on the CPU: the algorithmic byte and flop counts its roofline
objects use, counted here from the data layout and the stencil, and the
JSON contract of the reference arm (the CPU oracle), run on a small lattice."""
import json
import sys

import pytest

import bench


def test_bytes_per_site_from_the_layout():
    # 8 links (6 in the temporal gauge) + one input and one output spinor
    spinor = {0: 24 * 8, 1: 24 * 4, 2: 24 * 2 + 4, 3: 24 * 2 + 4, 4: 24 * 2 + 4}
    link12 = {1: 12 * 4, 2: 12 * 2, 3: 12 * 2, 4: 12 * 2}
    assert bench.bytes_per_site(0, 18) == 8 * 18 * 8 + 2 * spinor[0] == 1536
    assert bench.bytes_per_site(0, 18, tfix=True) == 6 * 18 * 8 + 2 * spinor[0] == 1248
    assert bench.bytes_per_site(0, 12) == 8 * 12 * 8 + 2 * spinor[0] == 1152
    for p in (1, 2, 3, 4):
        assert bench.bytes_per_site(p, 12) == 8 * link12[p] + 2 * spinor[p]
        assert bench.bytes_per_site(p, 12, tfix=True) == 6 * link12[p] + 2 * spinor[p]
        # App. A.2: 8 numbers instead of 12 reals per link
        assert bench.bytes_per_site(p, 12, tfix=True, recon8=True) == 6 * link12[p] * 8 // 12 + 2 * spinor[p]
    assert bench.bytes_per_site(2, 12) == 296 and bench.bytes_per_site(2, 12, tfix=True) == 248


def test_flops_per_site():
    # one SU(3) matrix on a two-spin half spinor: 2 x 3 rows x (3 complex
    # multiplies of 6 flops + 2 complex adds of 2 flops) = 132
    su3_half = 2 * 3 * (3 * 6 + 2 * 2)
    assert su3_half == 132
    assert bench.flops_per_site() == 1320
    assert bench.flops_per_site(tfix=True) == 1320 - 2 * su3_half


def test_reference_arm_json_contract(monkeypatch, capsys):
    small = dict(bench.WORKLOAD)
    small["dims"] = (4, 4, 4, 8)
    monkeypatch.setattr(bench, "WORKLOAD", small)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"])
    assert bench.main() in (0, None)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "solves/s"
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    # a step is the sampled part of a solve, timed as it ran; value extrapolates
    # it to whole solves by the stated factor
    cb0 = line["cpu_baseline"]
    assert line["ms_per_step"] == pytest.approx(1000.0 * cb0["sample_seconds"], rel=1e-3)
    assert line["value"] == pytest.approx(cb0["sample_iterations"] / (cb0["sample_seconds"] * cb0["full_solve_iterations"]),
                                          rel=1e-2)
    assert cb0["extrapolated"] and cb0["scale"] == pytest.approx(cb0["full_solve_iterations"] / cb0["sample_iterations"],
                                                                 rel=1e-3)
    assert line["config"]["workload"] == bench.WORKLOAD["workload"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_recorded_traffic_is_tied_to_the_kernel_sources(monkeypatch):
    """The ncu traffic the bench line reports belongs to the kernel revision it
    was captured on: with another source hash it is reported as null."""
    key = ("q16", 12, "24x24x24x64", True)
    monkeypatch.setattr(bench, "NCU_TRAFFIC_BYTES", {key: 1.0e8})
    monkeypatch.setattr(bench, "KERNEL_SOURCES_SHA", bench.kernel_sources_sha())
    assert bench.ncu_traffic(key) == 1.0e8
    assert bench.ncu_traffic(("q16", 12, "64x64x64x128", True)) is None
    monkeypatch.setattr(bench, "KERNEL_SOURCES_SHA", "0" * 16)
    assert bench.ncu_traffic(key) is None
