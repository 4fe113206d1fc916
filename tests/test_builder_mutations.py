"""Mutation check of the host tests of the product builder: every mistake
below, planted in a copy of the library sources, makes the builder-versus-
oracle table tests, the nesting test of the packed box codes or the KD
tree's box test in tests/test_abi_host.py fail, while the unmodified copy
passes them.  Each copy of the package is built into a temporary
directory and tested in a subprocess on the CPU (no GPU is visible to it);
the committed sources are never touched."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2308_16084_gb300"

# (name, file under csrc/, original text, planted text)
MUTATIONS = [
    ("filter sign flipped in the flooding core", "flood_core.h",
     "      gv[q] = len2(x - pv) - dist2 + eta;",
     "      gv[q] = dist2 - len2(x - pv) + eta;"),
    ("face Space-perp on the outer side", "builder.cpp",
     "        perp[np_++] = {-1.0 * m, -dot(m, pk) + delta, -20 - k};",
     "        perp[np_++] = {m, dot(m, pk) + delta, -20 - k};"),
    ("Region box lower corner not padded", "flood_core.h",
     "      box[d] = l;",
     "      box[d] = (float)blo[d];"),
    ("flood never leaves the seeds", "flood_core.h",
     "      if (env.mark(w, queue, tail)) {",
     "      if (false && env.mark(w, queue, tail)) {"),
    ("chunk codes without their two-code widening", "builder.cpp",
     "        cl[d] = a >= 2 ? a - 2 : 0;\n        ch[d] = std::min(kQMax, b + 2);",
     "        cl[d] = a;\n        ch[d] = b;"),
    ("super-chunk codes from its first chunk only", "builder.cpp",
     "      for (uint32_t k = c; k < ce; ++k) {\n        uint32_t cl[3], ch[3];",
     "      for (uint32_t k = c; k < c + 1; ++k) {\n        uint32_t cl[3], ch[3];"),
    ("chunk hull from its first entry only", "builder.cpp",
     "      for (uint32_t k = j; k < j + cnt; ++k)\n        for (int d = 0; d < 3; ++d) {\n"
     "          lo[d] = std::min(lo[d], all[k].box[d]);",
     "      for (uint32_t k = j; k < j + 1; ++k)\n        for (int d = 0; d < 3; ++d) {\n"
     "          lo[d] = std::min(lo[d], all[k].box[d]);"),
    ("KD children's boxes exported swapped", "builder.cpp",
     "    const double *c0 = &T.box[6 * (2 * i + 1)], *c1 = &T.box[6 * (2 * i + 2)];",
     "    const double *c0 = &T.box[6 * (2 * i + 2)], *c1 = &T.box[6 * (2 * i + 1)];"),
]

TESTS = "(tables_equal_oracle_tables and not random) or packed_codes or kd_tree_boxes"


def _host_tests_with_copy(base, name, fname, old, new):
    work = os.path.join(base, name.replace(" ", "_"))
    # the built objects come along with their times, so the copy's build
    # recompiles only what the planted mistake touches
    shutil.copytree(os.path.join(ROOT, PKG), os.path.join(work, PKG),
                    ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(os.path.join(ROOT, "include"), os.path.join(work, "include"))
    if fname is not None:
        src = os.path.join(work, PKG, "csrc", fname)
        text = open(src).read()
        assert text.count(old) == 1, name
        open(src, "w").write(text.replace(old, new))
    # CPU only: the copies never see a GPU
    env = {**os.environ, "PYTHONPATH": work + os.pathsep + ROOT, "CUDA_VISIBLE_DEVICES": ""}
    b = subprocess.run([sys.executable, os.path.join(work, PKG, "build.py")], cwd=work,
                       env=env, capture_output=True, text=True, timeout=900)
    assert b.returncode == 0, b.stdout + b.stderr
    where = subprocess.run([sys.executable, "-c",
                            f"import {PKG} as p; print(p._lib.LIB_PATH)"],
                           cwd=work, env=env, capture_output=True, text=True, timeout=300)
    assert where.stdout.strip().startswith(work), where.stdout + where.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "--import-mode=append", "-k", TESTS,
                        os.path.join(ROOT, "tests", "test_abi_host.py")],
                       cwd=work, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-1500:] + r.stderr[-1500:]


def test_every_planted_builder_mistake_fails_a_host_test(tmp_path):
    runs = [("unmodified", None, None, None)] + MUTATIONS
    with cf.ThreadPoolExecutor(4) as ex:
        res = list(ex.map(lambda m: _host_tests_with_copy(str(tmp_path), *m), runs))
    code, out = res[0]
    assert code == 0, "the unmodified copy must pass:\n" + out
    missed = [runs[i][0] for i in range(1, len(runs)) if res[i][0] != 1]
    assert not missed, f"mistakes no host test caught (or that crashed): {missed}\n" + \
        "\n".join(res[i][1] for i in range(1, len(runs)) if res[i][0] != 1)
