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
