"""Mutation check of the oracle's pins: every mistake below, planted in a
copy of oracle/p2m_oracle.c, makes the pin suite (tests/test_oracle_pins.py)
fail, while the unmodified copy passes it.  The copies live in a temporary
directory and are imported in subprocesses; the committed oracle is never
touched."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text, planted text): each original occurs exactly once
MUTATIONS = [
    ("edge gate past the far end",
     "  if (!(t > 0.0 && t < 1.0)) return 0;",
     "  if (!(t > 0.0 && t < 1.2)) return 0;"),
    ("face barycentric weights swapped",
     "  c->bw[0] = 1.0 - s - t; c->bw[1] = s; c->bw[2] = t;",
     "  c->bw[0] = 1.0 - s - t; c->bw[1] = t; c->bw[2] = s;"),
    ("face Space-perp on the outer side",
     "      pl[4 * k + 0] = -mm[0]; pl[4 * k + 1] = -mm[1]; pl[4 * k + 2] = -mm[2];\n"
     "      pl[4 * k + 3] = -dot3(mm, a) + m->delta;",
     "      pl[4 * k + 0] = mm[0]; pl[4 * k + 1] = mm[1]; pl[4 * k + 2] = mm[2];\n"
     "      pl[4 * k + 3] = dot3(mm, a) + m->delta;"),
    ("filter sign flipped",
     "  return dist2(x, pv) - prim_dist2(dp, x) + m->eta;",
     "  return prim_dist2(dp, x) - dist2(x, pv) + m->eta;"),
    ("KD tree prunes too early",
     "  if (kd_box_d2(m, node, q) > *bd2) return;",
     "  if (kd_box_d2(m, node, q) > 0.25 * *bd2) return;"),
    ("flood never leaves the seeds",
     "      if (T->stamp[w] != mark) {",
     "      if (0) {"),
    ("edge slab missing its far endpoint plane",
     "  pl[4] = u[0]; pl[5] = u[1]; pl[6] = u[2]; pl[7] = dot3(u, b) + m->delta;\n  k = 2;",
     "  k = 1;"),
    ("Region box not padded",
     "    box[d] = lo[d] - m->delta;\n    box[3 + d] = hi[d] + m->delta;",
     "    box[d] = lo[d];\n    box[3 + d] = hi[d];"),
    ("Region box over the whole polytope",
     "      if (g0 > 0.0) { keep = 1; GROW(x0); }",
     "      if (g0 > 0.0) keep = 1;\n      GROW(x0);"),
    ("Region box without the edge crossings",
     "          GROW(xc);\n        }\n      }",
     "          (void)xc;\n        }\n      }"),
    ("ties between types reversed",
     "  if (a->type != b->type) return a->type < b->type;",
     "  if (a->type != b->type) return a->type > b->type;"),
    ("ties between ids reversed",
     "  return a->id < b->id;\n}",
     "  return a->id > b->id;\n}"),
    ("second-best distance kept from earlier bests only",
     "    else if (cand_better(&c, &sec)) sec = c;         \\",
     "    else if (0) sec = c;                             \\"),
    ("KD tree prunes a subtree at equal distance",
     "  if (kd_box_d2(m, node, q) > *bd2) return;",
     "  if (kd_box_d2(m, node, q) >= *bd2) return;"),
    ("widened cells' bisectors not pushed out",
     "    bisector_plane(m, (int32_t)i, x->nbs[i][j], m->delta, pl);",
     "    bisector_plane(m, (int32_t)i, x->nbs[i][j], 0.0, pl);"),
    ("widened cells' domain not grown",
     "  for (int d = 0; d < 3; ++d) { lo[d] = m->dlo[d] - m->delta; hi[d] = m->dhi[d] + m->delta; }",
     "  for (int d = 0; d < 3; ++d) { lo[d] = m->dlo[d]; hi[d] = m->dhi[d]; }"),
]


def _pins_with_oracle_copy(base, name, old, new):
    """Run the pin suite against a copy of the oracle with `old` replaced by
    `new` (none when old is None).  Returns (pytest exit code, output)."""
    work = os.path.join(base, name.replace(" ", "_"))
    dst = os.path.join(work, "oracle")
    shutil.copytree(os.path.join(ROOT, "oracle"), dst,
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    src = os.path.join(dst, "p2m_oracle.c")
    text = open(src).read()
    if old is not None:
        assert text.count(old) == 1, name
        open(src, "w").write(text.replace(old, new))
    # CPU only: the copies never see a GPU
    env = {**os.environ, "PYTHONPATH": work + os.pathsep + ROOT, "CUDA_VISIBLE_DEVICES": ""}
    where = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.__file__)"],
                           cwd=work, env=env, capture_output=True, text=True, timeout=300)
    assert where.stdout.strip().startswith(dst), where.stdout + where.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "--import-mode=append", os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=work, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-1500:] + r.stderr[-1500:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    runs = [("unmodified", None, None)] + MUTATIONS
    with cf.ThreadPoolExecutor(max(4, min(8, os.cpu_count() or 4))) as ex:
        res = list(ex.map(lambda m: _pins_with_oracle_copy(str(tmp_path), *m), runs))
    code, out = res[0]
    assert code == 0, "the unmodified copy must pass the pins:\n" + out
    missed = [runs[i][0] for i in range(1, len(runs)) if res[i][0] != 1]
    assert not missed, f"mistakes no pin caught (or that crashed): {missed}\n" + \
        "\n".join(res[i][1] for i in range(1, len(runs)) if res[i][0] != 1)
