"""bench.py's contract on the CPU: the reference arm (the FP64 oracle timed
on the host cores) prints one JSON line with every key the benchmark line
needs, and the product arm fails loudly without a GPU (no CPU fallback)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_complete_line():
    # the full-size arm builds the oracle's tables of the level-8 mesh
    # (minutes); the same code on the level-4 mesh of the same recipe
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "1", "--level", "4",
             "--queries", "200000")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e", "impl"):
        assert k in j, k
    assert j["impl"] == "reference"
    assert j["value"] > 0 and j["unit"] == "queries/s" and j["higher_is_better"] is True
    assert (j["n_gpus"], j["steps"], j["warmup"]) == (1, 1, 1)
    assert j["vs_baseline"] is None and j["data"] == "synthetic"
    assert "workload" in j["config"] and j["config"]["reduced"] is True
    assert "P2M query" in j["cpu_baseline"]["sample"]
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == j["value"]
    assert j["e2e"] == {"value": j["value"], "unit": j["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_product_arm_needs_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _run("--steps", "3", "--warmup", "3", "--level", "2", "--queries", "1000",
             "--no-cpu-baseline", timeout=300)
    assert r.returncode != 0
    assert not [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]


def test_algorithmic_bytes_model():
    """The roofline's byte model: B_q = 12 + 20 + 16 N_kdt + 8 + 28 L_scan
    + 24 T_e + 36 T_f per query, and the dominant (list) kernel's share is
    all of it but the nearest-vertex search's 16 N_kdt."""
    sys.path.insert(0, ROOT)
    import bench
    c = {"nodes": 0, "points": 179, "entries": 159, "edges": 51, "faces": 62, "chunks": 111}
    bq, bnn, blist = bench.algorithmic_bytes(c, 10)
    assert abs(bq - (12 + 20 + 16 * 17.9 + 8 + 28 * 15.9 + 24 * 5.1 + 36 * 6.2)) < 1e-9
    assert abs(blist - (bq - 16 * 17.9)) < 1e-9
    assert abs(bnn - (12 + 16 * 17.9)) < 1e-9


def test_oracle_sample_is_seeded_and_sorted():
    sys.path.insert(0, ROOT)
    import bench
    a = bench.oracle_sample(10_000_000, 5000)
    b = bench.oracle_sample(10_000_000, 5000)
    assert (a == b).all() and (a[1:] > a[:-1]).all() and a.max() < 10_000_000


def test_clock_samples_summary():
    """The clocks object: median SM clock under load, the highest maximum
    clock reported, and every throttle reason seen active in any sample;
    header, unit or malformed lines are skipped."""
    sys.path.insert(0, ROOT)
    import bench
    na, act = "Not Active", "Active"
    lines = [
        "index, clocks.sm [MHz], clocks.max.sm [MHz], power.draw [W], ...",
        f"0, 2070, 2070, 900.5, 0x0, {na}, {na}, {na}, {na}",
        f"0, 1980, 2070, 1400.0, 0x4, {na}, {na}, {na}, {act}",
        f"0, 2070, 2070, 1100.2, 0x0, {na}, {na}, {na}, {na}",
        "0, [N/A], 2070, 0, 0x0, N/A, N/A, N/A, N/A",
        "garbage",
    ]
    s = bench.ClockSampler.summarise(lines)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    hot = bench.ClockSampler.summarise([f"0, 1500, 2070, 1300, 0x8, {na}, {act}, {act}, {na}"])
    assert hot["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler.summarise([])["sm_mhz"] is None


def test_kernels_per_step_counts_the_launches_of_a_call():
    """gpu_launches: the sort (count, three scans, scatter; one copy of the
    queries in their own order when the sort is off), then either the
    one-pass kernel, which writes the outputs itself, or per concurrent
    range the nn pass, three scans, the vertex scatter and the list pass,
    and then the output write.  A range holds at least 2^18 queries."""
    sys.path.insert(0, ROOT)
    import bench
    two_pass = {"sort_bits": 12, "group_by_vertex": 1, "warp_cooperative": 0, "streams": 2}
    assert bench.kernels_per_step(two_pass, 10_000_000) == 5 + 12 + 1
    assert bench.kernels_per_step(two_pass, 100_000) == 5 + 6 + 1
    assert bench.kernels_per_step(dict(two_pass, streams=1), 10_000_000) == 12
    one_pass = {"sort_bits": 0, "group_by_vertex": 0}
    assert bench.kernels_per_step(one_pass, 100_000) == 2
    assert bench.kernels_per_step(dict(two_pass, warp_cooperative=1), 10_000_000) == 6
