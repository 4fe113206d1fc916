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
