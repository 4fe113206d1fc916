"""The product builder and the oracle under AddressSanitizer (with leak
checking) and UBSan, on the host.  tests/builder_host_check.cpp builds each
mesh on the host, again through stand-ins for the device services
(brute-force certification searches, the device kernel's warp flooding run
lane by lane on the host) and compares the layouts, then injects an
allocation failure into each build stage; tests/oracle_host_check.c runs
the oracle's tables, brute force and queries.  Any sanitizer report fails
the run."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import datagen as dg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2308_16084_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("asan") / "builder_host_check")
    cmd = ["g++", "-O1", "-g", "-std=c++17", "-pthread", "-ffp-contract=off",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "builder_host_check.cpp"),
           os.path.join(CSRC, "builder.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


@pytest.fixture(scope="module")
def oracle_checker(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path_factory.mktemp("asan_oracle") / "oracle_host_check")
    cmd = ["gcc", "-O1", "-g", "-std=gnu11", "-pthread", "-ffp-contract=off",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-I", os.path.join(ROOT, "oracle"), os.path.join(ROOT, "tests", "oracle_host_check.c"),
           os.path.join(ROOT, "oracle", "p2m_oracle.c"), "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def _write(m, path):
    segs = m.meta.get("segs")
    S = np.zeros((0, 2), np.int32) if segs is None else np.asarray(segs, np.int32)
    with open(path, "wb") as f:
        np.array([m.verts.shape[0], m.tris.shape[0], S.shape[0]], np.int64).tofile(f)
        np.ascontiguousarray(m.verts, np.float32).tofile(f)
        np.ascontiguousarray(m.tris, np.int32).tofile(f)
        np.ascontiguousarray(S, np.int32).tofile(f)
        np.array([m.domain_scale, m.domain_margin], np.float64).tofile(f)


@pytest.mark.parametrize("name", ["sphere", "soup", "mixed", "fan"])
def test_builder_under_sanitizers(checker, name, tmp_path):
    m = {"sphere": lambda: dg.workload(0, n_queries=10),
         "soup": lambda: dg.soup_workload("penetrating", level=2, n_queries=10),
         "mixed": lambda: dg.mixed_workload(mesh_level=2, wire_level=1, n_queries=10),
         "fan": lambda: dg.high_valence_fan(120)}[name]()
    path = str(tmp_path / "mesh.bin")
    _write(m, path)
    r = subprocess.run([checker, path], capture_output=True, text=True, timeout=900,
                       env={**os.environ, "ASAN_OPTIONS": "detect_leaks=1"})
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), \
        r.stdout[-2000:] + r.stderr[-3000:]


@pytest.mark.parametrize("name", ["sphere", "mixed", "fan"])
def test_oracle_under_sanitizers(oracle_checker, name, tmp_path):
    m = {"sphere": lambda: dg.workload(0, n_queries=10, level=2),
         "mixed": lambda: dg.mixed_workload(mesh_level=2, wire_level=1, n_queries=10),
         "fan": lambda: dg.high_valence_fan(60)}[name]()
    path = str(tmp_path / "mesh.bin")
    _write(m, path)
    r = subprocess.run([oracle_checker, path], capture_output=True, text=True, timeout=900,
                       env={**os.environ, "ASAN_OPTIONS": "detect_leaks=1"})
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), \
        r.stdout[-2000:] + r.stderr[-3000:]
