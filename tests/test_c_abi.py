"""include/p2m.h is a C header: a plain C99 program (tests/c_abi_host.c)
compiles against it with -pedantic -Werror, links libp2m.so and runs the
host-side calls without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c99_client_builds_and_runs(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2308_16084_gb300 import build as b
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "c_abi_host")
    libdir = os.path.dirname(b.LIB)
    cmd = ["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_abi_host.c"),
           "-o", exe, "-L", libdir, "-lp2m", f"-Wl,-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe, str(tmp_path / "m.p2m")], capture_output=True, text=True,
                       timeout=120, env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr


def test_build_recompiles_what_changed_and_every_object_of_another_machine(tmp_path):
    """The package build reuses an object only while it is newer than its
    source and every header the source includes, and only on the machine
    type that compiled it: a copy of the tree carrying another
    architecture's objects is rebuilt whole."""
    import importlib.util
    import __graft_entry__
    __graft_entry__.build()
    pkg = os.path.join(tmp_path, "paper_2308_16084_gb300")
    shutil.copytree(os.path.join(ROOT, "paper_2308_16084_gb300"), pkg,
                    ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(os.path.join(ROOT, "include"), os.path.join(tmp_path, "include"))
    spec = importlib.util.spec_from_file_location("p2m_build_copy", os.path.join(pkg, "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    objs = {s: os.path.join(b.OUT, s + ".o") for s in b._sources()}

    def times():
        return {s: os.path.getmtime(o) for s, o in objs.items()}

    assert not b._stale()
    t0 = times()
    os.utime(os.path.join(b.CSRC, "pack_core.h"))  # included by pack.cu only
    b.build()
    t1 = times()
    assert [s for s in objs if t1[s] != t0[s]] == ["pack.cu"]
    with open(b.STAMP, "w") as f:
        f.write("another-machine\n")
    assert b._stale()
    b.build()
    t2 = times()
    assert all(t2[s] > t1[s] for s in objs)
    assert not b._stale()
