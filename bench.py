#!/usr/bin/env python3
"""Benchmark of the point-to-mesh query stage (P2M, Alg. A.2) on GB300.

One step = one pass of the whole query path (sort of the queries, nearest
vertex, interception-list scan with the Region-box filter, edge and face
tests, minimum, outputs in the caller's order) over one batch of synthetic
queries.  The headline is workload 1: the 1,310,720-triangle displaced
icosphere with 10M uniform queries.  The same JSON line (rank 0) also
carries the other four workloads, each with its own CUDA-event timing,
clocks, roofline and end-to-end figure:
  configs                     workloads 0 and 2: plain forward on the small
                              noisy icosphere and on the 2.1M-triangle
                              jittered height field;
  fwd_bwd                     workload 3: forward+backward against forward;
  batched                     workload 4: 64 meshes in one CUDA-graph launch
                              against 64 per-mesh launches.
cpu_baseline is the FP64 oracle's own P2M query (Alg. A.2, tables built
beforehand and not timed) on a seeded sample of workload 1, on all host
cores; its tables are built by a spawned process while the GPU runs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times that oracle query alone (host cores, rank 0), on the
same workload, metric and config.  For N > 1 (torchrun) every rank runs an
independent replica of the headline (the query path has no exchange step):
value = all ranks' queries / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time
import traceback

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import datagen as dg  # noqa: E402

METRIC = "point-to-mesh queries/sec (1.3M tris) + HBM roofline %; batched & fwd+bwd vs plain"
UNIT = "queries/s"
WORKLOAD = 1
L2_BYTES = 129 * 1024 * 1024


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=2_000_000,
                    help="queries of the seeded sample the CPU oracle's P2M query times")
    ap.add_argument("--cpu-bf-sample", type=int, default=1024,
                    help="queries of the sample the CPU brute force times")
    ap.add_argument("--cpu-timeout", type=float, default=1500.0,
                    help="seconds to wait for the CPU oracle's tables after the GPU work")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pipe-depth", type=int, default=8,
                    help="slots of the pipelined host API in the end-to-end figure")
    ap.add_argument("--only", default=None,
                    choices=["headline", "cfg0", "cfg2", "fwd_bwd", "batched"],
                    help="measure one part only (profiling runs)")
    ap.add_argument("--level", type=int, default=None, help="smaller mesh (profiling only)")
    ap.add_argument("--queries", type=int, default=None, help="fewer queries (profiling only)")
    ap.add_argument("--workload", type=int, default=None, choices=[3, 4],
                    help="shorthand for --only fwd_bwd (3) or --only batched (4)")
    ap.add_argument("--tuning", default=None,
                    help="fixed p2m_tuning fields as JSON (profiling runs with --no-autotune)")
    ap.add_argument("--sweep", action="store_true",
                    help="extra workloads: mesh resolution, query box, soups, good and poor "
                         "triangulations, mixed primitives, R-tree levels")
    ap.add_argument("--list-stats", action="store_true",
                    help="interception-list statistics of the workloads' tables (host build)")
    ap.add_argument("--layout", default=None,
                    help="load the built layout from this file if it exists, else build and "
                         "save it there")
    args = ap.parse_args(argv)
    if args.workload is not None and args.only is None:
        args.only = {3: "fwd_bwd", 4: "batched"}[args.workload]
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args):
    return dg.workload(WORKLOAD, n_queries=args.queries, level=args.level)


def config_of(m, args):
    """The workload the line is quoted on: the same dict in both arms."""
    c = {"workload": m.name, "mesh": "icosphere subdivided 8x, radial displacement 0.2",
         "n_tris": int(m.tris.shape[0]), "n_verts": int(m.verts.shape[0]),
         "n_queries_per_gpu": int(m.queries.shape[0]),
         "query_distribution": "uniform in bbox scaled 1.5x",
         "domain": f"bbox x{m.domain_scale} + {m.domain_margin} diag",
         "l2": "inputs larger than L2 (the 3.5 GB layout and 120 MB of queries per step), "
               "no flush"}
    if args.level is not None or args.queries is not None:
        c["reduced"] = True
    return c


def timed(fn, steps, stream, flush=None):
    """Device milliseconds of `steps` calls of fn, CUDA events on `stream`.
    With `flush` (a device buffer larger than L2), the buffer is rewritten
    between steps, outside the events, and the per-step times are summed."""
    import torch
    torch.cuda.synchronize()
    if flush is None:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for k, (a, b) in enumerate(evs):
        flush.fill_(k & 1)
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs)


def guarded(fn, *a, **kw):
    """Run one part of the measurement; a failure is reported in its place
    instead of costing the whole line."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001  (reported, not hidden)
        traceback.print_exc(file=sys.stderr)
        return {"error": f"{type(e).__name__}: {e}"[:500]}


# ----------------------------------------------------------------- oracle arm

def _oracle_worker(conn, level, n_queries, threads):
    """Spawned process: builds the FP64 oracle's tables of workload 1 (the
    Delaunay-neighbour Voronoi cells, then the flooding of Alg. 1), reports
    the build, then on request times the oracle's P2M query (Alg. A.2 with
    the Region-box filter) and its brute force on seeded samples."""
    try:
        os.nice(5)
    except OSError:
        pass
    try:
        import oracle
        m = dg.workload(WORKLOAD, n_queries=n_queries, level=level)
        t0 = time.perf_counter()
        # two cores left to the GPU side while the tables build beside its
        # measurements (its end-to-end loop and the builder's host threads);
        # the timed queries below take all of them
        o = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin,
                              threads=max(1, threads - 2), voronoi="delaunay")
        build_s = time.perf_counter() - t0
        conn.send(("built", {"build_s": round(build_s, 1), "qhull_s": round(o.delaunay_s, 1),
                             "table_entries": o.n_entries, "times_ms": o.times_ms}))
        while True:
            msg = conn.recv()
            if msg[0] == "stop":
                return
            _, sample, bf_sample, per_step = msg
            conn.send(("timed", time_oracle(o, m, sample, bf_sample, threads, per_step)))
    except Exception as e:  # noqa: BLE001
        conn.send(("error", f"{type(e).__name__}: {e}"[:500]))


def oracle_sample(n_total, k, seed=16084):
    """Seeded sample of k query indices (sorted) out of n_total."""
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(10)[9])
    k = min(k, n_total)
    return np.sort(rng.choice(n_total, k, replace=False))


def time_oracle(o, m, sample, bf_sample, threads, per_step=None):
    """Times the oracle's P2M query on a seeded sample of the workload's
    queries (all threads), and its brute force on the first bf_sample of
    them.  per_step: (warmup, steps, queries per step) for the reference
    arm, which times that many steps of the P2M query instead."""
    idx = oracle_sample(m.queries.shape[0], sample)
    q = m.queries[idx]
    o.query(q[:2000], use_boxes=True, threads=threads)  # warm-up: pages, caches
    out = {"threads": threads}
    if per_step:
        w, k, per = per_step
        for s in range(w):
            o.query(q[(s * per) % len(q):][:per], use_boxes=True, threads=threads)
        t0 = time.perf_counter()
        done = 0
        for s in range(k):
            a = ((w + s) * per) % len(q)
            qq = q[a:a + per]
            o.query(qq, use_boxes=True, threads=threads)
            done += qq.shape[0]
        out["steps_s"] = time.perf_counter() - t0
        out["steps_queries"] = done
        return out
    t0 = time.perf_counter()
    r = o.query(q, use_boxes=True, threads=threads, counters=True)
    dt = time.perf_counter() - t0
    c = r["counters"].mean(0)
    out.update({"n": int(q.shape[0]), "s": dt,
                "work_per_query": {"kdt_nodes": float(c[0]), "entries": float(c[1]),
                                   "edges": float(c[2]), "faces": float(c[3])}})
    nb = min(bf_sample, q.shape[0])
    t0 = time.perf_counter()
    o.bruteforce(q[:nb], threads=threads)
    out["bf_n"] = int(nb)
    out["bf_s"] = time.perf_counter() - t0
    return out


class OracleWorker:
    """The oracle's table build of workload 1 in a spawned process, started
    before the first GPU call so that it overlaps the GPU work."""

    def __init__(self, args, threads):
        ctx = mp.get_context("spawn")
        self.conn, child = ctx.Pipe()
        self.proc = ctx.Process(target=_oracle_worker,
                                args=(child, args.level, args.queries, threads), daemon=True)
        self.proc.start()
        self.threads = threads
        self.built = None

    def wait_built(self, timeout):
        if self.built is None:
            if not self.conn.poll(timeout):
                raise TimeoutError(f"oracle tables not built within {timeout:.0f} s")
            tag, info = self.conn.recv()
            if tag != "built":
                raise RuntimeError(f"oracle worker: {info}")
            self.built = info
        return self.built

    def time(self, sample, bf_sample, per_step=None, timeout=1200):
        self.conn.send(("go", sample, bf_sample, per_step))
        if not self.conn.poll(timeout):
            raise TimeoutError("oracle query timing did not finish")
        tag, info = self.conn.recv()
        if tag != "timed":
            raise RuntimeError(f"oracle worker: {info}")
        return info

    def close(self):
        try:
            self.conn.send(("stop",))
        except (OSError, BrokenPipeError):
            pass
        self.proc.join(timeout=30)
        if self.proc.is_alive():
            self.proc.kill()


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline_of(res, built, n_total):
    per_q = res["s"] / res["n"]
    v = res["n"] / res["s"]
    return {"value": v, "unit": UNIT, "cores": res["threads"], "kind": "oracle",
            "sample": f"seeded {res['n']} of the {n_total} queries; the FP64 oracle's P2M query "
                      "(Alg. A.2: KD-tree nearest vertex, interception list, Region-box "
                      "filter, gated edge and face distances) with its tables built "
                      f"beforehand ({built['build_s']} s, not timed); value extrapolated "
                      "from the sample",
            "us_per_query_per_core": per_q * 1e6 * res["threads"],
            "extrapolated": True, "cpu_model": cpu_model(),
            "oracle_build_s": built["build_s"], "oracle_table_entries": built["table_entries"],
            "paper_method_work_per_query": res["work_per_query"]}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    m = workload(args)
    threads = os.cpu_count() or 1
    worker = OracleWorker(args, threads)
    try:
        built = worker.wait_built(args.cpu_timeout)
        per = max(1000, min(200_000, args.cpu_sample // max(1, args.steps + args.warmup)))
        res = worker.time(per * (args.steps + args.warmup), 0,
                          per_step=(args.warmup, args.steps, per))
    finally:
        worker.close()
    dt = res["steps_s"]
    v = res["steps_queries"] / dt
    sample = (f"{per} queries per step from a seeded sample of the {m.queries.shape[0]} "
              "queries; the FP64 oracle's P2M query (Alg. A.2 with the Region-box filter) "
              f"on tables built beforehand ({built['build_s']} s, not timed)")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "hardware": f"host cores only ({threads} threads, {cpu_model()}): rank 0 runs the "
                        "oracle, the GPUs stay idle",
            "config": config_of(m, args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons (read only)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        return self.summarise(self.lines)

    @staticmethod
    def summarise(lines):
        """Median and maximum SM clock and the throttle reasons seen active
        in nvidia-smi's CSV lines (FIELDS, no header, no units); lines that
        do not parse are skipped."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- our arm

def kernel_hash():
    """Digest of the device sources (kernels and the box decoding they
    include): a stored ncu figure is used only while it matches."""
    h = hashlib.sha256()
    for name in ("kernels.cu", "kernels.h", "quant.h"):
        with open(os.path.join(ROOT, "paper_2308_16084_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, n_queries):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    profiles/<kernel>_dram.json, if it was taken on the current kernel
    source; else None."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_dram.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    if d.get("kernel_sha") != kernel_hash() or not d.get("dram_bytes_per_query"):
        return None
    return d["dram_bytes_per_query"] * n_queries


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def phase_bytes(c, n, out_bytes=21):
    """Algorithmic bytes one query touches in each kernel, from the record
    sizes of the layout and the work counters.
      nearest-vertex pass: sorted query 16 B, (vertex, rank) out 8 B,
        seed-grid cell 4 B, 48 B per KD internal node (backtracking only),
        16 B per vertex record examined (seed, Voronoi neighbours);
      list pass: regrouped query 16 B + vertex 4 B, nearest-vertex record
        16 B, three CSR ranges 24 B, 16 B per super/chunk box tested, 16 B
        per list entry scanned, 32 B per edge and 48 B per face tested,
        32-byte result record out;
      output write: the 32-byte record in, the requested outputs out
        (out_bytes: 21 B for dist, closest, id and type)."""
    nn = (16 + 8 + 4) * n + 48 * c["nodes"] + 16 * c["points"]
    lst = (16 + 4 + 16 + 24 + 32) * n + 16 * c.get("chunks", 0) + 16 * c["entries"] + \
        32 * c["edges"] + 48 * c["faces"]
    return nn / n, lst / n, 32 + out_bytes


def algorithmic_bytes(c, n):
    """Bytes per query the method itself touches, with fixed minimal record
    sizes, from the work counters (c: totals over n queries):
        B_q = 12 (query) + 20 (distance, closest point, primitive)
              + 16 N_kdt (KD nodes / vertex records visited) + 8 (CSR range)
              + 28 L_scan (4 B entry id + 24 B Region box per entry scanned)
              + 24 T_e (two endpoints per edge tested)
              + 36 T_f (three vertices per face tested).
    Returns (whole query, nearest-vertex part, list part); the list part is
    everything but the 16 N_kdt of the nearest-vertex search."""
    n_kdt = (c["nodes"] + c["points"]) / n
    nn = 12 + 16 * n_kdt
    lst = 12 + 20 + 8 + 28 * c["entries"] / n + 24 * c["edges"] / n + 36 * c["faces"] / n
    return 12 + 20 + 16 * n_kdt + 8 + 28 * c["entries"] / n + 24 * c["edges"] / n + \
        36 * c["faces"] / n, nn, lst


def kernels_per_step(tuning, n=0):
    """This library's kernels per query call: the sort (count, 3 scan kernels,
    scatter), then either the one-pass kernel or, per concurrent range of the
    sorted queries (tuning field streams, ranges of >= 2^18), the nn pass, 3
    scan kernels, the vertex scatter and the list pass, and one output
    write."""
    sort = 5 if tuning["sort_bits"] > 0 else 1
    if tuning.get("group_by_vertex") and not tuning.get("warp_cooperative"):
        ranges = max(1, min(tuning.get("streams", 1), n >> 18))
        return sort + 6 * ranges + 1
    return sort + 1


def max_over_ranks(values, dist):
    """Element-wise maximum of per-rank floats over all ranks: the slowest
    replica sets each time.  dist is torch.distributed (NCCL or gloo) or
    None for one process."""
    if dist is None:
        return list(values)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def share_layout(rank, world, build, load, path, dist):
    """Rank 0 builds the layout and saves it to `path`; the other replicas
    load it after a barrier (the query path has no exchange step, so this
    file is the only thing the replicas share)."""
    mesh = None
    if rank == 0:
        mesh = build()
        if world > 1:
            mesh.save(path)
    if world > 1:
        dist.barrier()
        if rank != 0:
            mesh = load(path)
        dist.barrier()
    return mesh


def replica_throughput(units_per_rank, steps, world, seconds):
    """Whole-job rate of N replicas: all ranks' units over the slowest
    rank's time."""
    return units_per_rank * steps * world / seconds


def forward_roofline(mesh, q, n, tsum, ms_step, steps):
    """Roofline object of the dominant kernel of the forward query: the
    algorithmic bytes of the kernel (the byte model of algorithmic_bytes,
    from the work counters) over its mean live duration (CUDA events on the
    launching stream over the timed steps), against the measured copy
    bandwidth; with the whole step's figure, the layout's actual record
    sizes and, where an ncu capture of the current source exists, DRAM."""
    cnt = mesh.counters(q)
    nn_b, list_b, out_b = phase_bytes(cnt, n)
    calls = max(1, tsum["calls"])
    tune = mesh.tuning
    grouped = bool(tune["group_by_vertex"]) and not tune["warp_cooperative"]
    phases = {"sort_ms": tsum["sort_ms"] / calls, "nn_pass_ms": tsum["nn_ms"] / calls,
              "regroup_ms": tsum["regroup_ms"] / calls, "list_pass_ms": tsum["list_ms"] / calls,
              "output_ms": tsum["output_ms"] / calls}
    bq, bq_nn, bq_list = algorithmic_bytes(cnt, n)
    if grouped:
        cand = [("k_nn_pass", phases["nn_pass_ms"], bq_nn, nn_b),
                ("k_list_pass", phases["list_pass_ms"], bq_list, list_b),
                ("k_unpack", phases["output_ms"], 0.0, out_b)]
    else:
        cand = [("k_query", phases["list_pass_ms"], bq, nn_b + list_b - 32 + 21)]
    kname, kms, kbytes, ktouched = max(cand, key=lambda c: c[1])
    peak, src = peaks()
    achieved = kbytes * n / (kms / 1e3) / 1e9
    step_achieved = bq * n * steps / (ms_step * steps / 1e3) / 1e9
    traffic = measured_traffic(kname, n)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured"
            else "fallback 6.8 TB/s",
            "kernel": kname, "kernel_ms": kms, "bytes_per_query": kbytes,
            "bytes_model": "B_q = 12 + 20 + 16 N_kdt + 8 + 28 L_scan + 24 T_e + 36 T_f "
                           "(the method's own touches at minimal record sizes, from the "
                           "work counters); the dominant kernel is charged all of B_q but "
                           "the 16 N_kdt of the nearest-vertex search",
            "bytes_per_query_step": bq,
            "achieved_step": step_achieved, "frac_step": step_achieved / peak,
            "touched_bytes_per_query": ktouched,
            "touched_frac": ktouched * n / (kms / 1e3) / 1e9 / peak,
            "note": "achieved and frac: algorithmic bytes of the dominant kernel over its "
                    "live CUDA-event duration; frac_step: all of B_q over the whole step; "
                    "touched_frac: the layout's actual record sizes (R-tree boxes "
                    "included); dram_frac: ncu DRAM bytes of the same launch over its "
                    "duration.  After the regrouping by nearest vertex the lanes of a warp "
                    "share one list, so most algorithmic bytes are served by L1/L2 and frac "
                    "can exceed 1 while dram_frac stays low",
            "phases": phases, "bytes_per_query_by_kernel": {"k_nn_pass": bq_nn,
                                                            "k_list_pass": bq_list},
            "touched_bytes_per_query_by_kernel": {"k_nn_pass": nn_b, "k_list_pass": list_b,
                                                  "k_unpack": out_b},
            "work_per_query": {k: v / n for k, v in cnt.items()}}
    if traffic:
        roof["dram_achieved"] = traffic / (kms / 1e3) / 1e9
        roof["dram_frac"] = roof["dram_achieved"] / peak
    return roof


def phase_times(mesh, q, out, steps, flush=None):
    """The phases of `steps` queries, CUDA events per phase on the launching
    stream (a separate pass: the timed region runs without them); with
    `flush`, L2 is rewritten between the queries as in the timed region."""
    import torch
    mesh.set_timing(True)
    mesh.timing_summary()
    for k in range(steps):
        if flush is not None:
            flush.fill_(k & 1)
        mesh.query(q, out=out)
    torch.cuda.synchronize()
    tsum = mesh.timing_summary()
    mesh.set_timing(False)
    return tsum


def out_buffers(torch, n):
    return {"dist": torch.empty(n, device="cuda"),
            "prim_id": torch.empty(n, dtype=torch.int32, device="cuda"),
            "closest": torch.empty(n, 3, device="cuda"),
            "prim_type": torch.empty(n, dtype=torch.uint8, device="cuda")}


def concurrent_steps(mesh, q, n, steps, depth):
    """The same steps device-resident, issued round robin on the `depth`
    slots of a pipe (p2m_pipe_submit_device: each slot its own stream,
    scratch and outputs), so that the kernels of neighbouring steps overlap,
    as they do in the pipelined end-to-end figure.  CUDA events on the
    launching stream: every step waits for the start event, and the stream
    joins every slot (p2m_pipe_join) before the end event."""
    import torch
    cur = torch.cuda.current_stream()
    outs = [out_buffers(torch, n) for _ in range(depth)]
    pipe = mesh.pipeline(n, depth=depth)
    for k in range(2 * depth):
        pipe.submit_device(q, outs[k % depth])
    pipe.join()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for k in range(steps):
        pipe.submit_device(q, outs[k % depth])
    pipe.join()
    e1.record(cur)
    torch.cuda.synchronize()
    pipe.close()
    ms = e0.elapsed_time(e1)
    return {"value": n * steps / (ms / 1e3), "unit": UNIT, "slots": depth,
            "ms_per_step": ms / steps,
            "api": "p2m_pipe_submit_device round robin on the slots, p2m_pipe_join"}


def pipe_e2e(mesh, m, steps, dist=None, depth=2):
    """End to end through the host APIs on pinned host buffers: every step
    copies its queries in and all four outputs out inside the timed region.
    Serial: p2m_query_host (copy in, query, copy out, synchronise).
    Pipelined: p2m_pipe_submit on `depth` slots, so one step's copies overlap
    the other step's kernels; the clock stops when the last step's results
    are in host memory.  Returns the two times in seconds."""
    import torch
    n = m.queries.shape[0]
    qh = torch.from_numpy(m.queries).pin_memory()
    outs_h = [(torch.empty(n, dtype=torch.float32).pin_memory(),
               torch.empty(n, dtype=torch.int32).pin_memory(),
               torch.empty(n, 3, dtype=torch.float32).pin_memory(),
               torch.empty(n, dtype=torch.uint8).pin_memory()) for _ in range(depth)]
    for _ in range(2):
        mesh.query_host(qh, *outs_h[0])
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        mesh.query_host(qh, *outs_h[0])
    serial_s = time.perf_counter() - t0
    pipe = mesh.pipeline(n, depth=depth)
    for k in range(depth):
        pipe.submit(qh, *outs_h[k])
    pipe.wait()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(steps):
        pipe.submit(qh, *outs_h[k % depth])
    pipe.wait()
    e2e_s = time.perf_counter() - t0
    pipe.close()
    return e2e_s, serial_s


def measure_forward(pg, m, args, local, *, steps, warmup, flush=None, dist=None,
                    world=1, layout=None):
    """Build, autotune and time the plain forward query of one workload:
    device-resident steps (CUDA events), per-phase times, roofline, and the
    end-to-end figure through the pipelined host API."""
    import torch
    rank = dist.get_rank() if dist else 0
    n = m.queries.shape[0]
    t0 = time.perf_counter()
    if layout and os.path.exists(layout):
        mesh = pg.P2M.load(layout)
    else:
        def build_and_keep():
            mh = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale,
                        domain_margin=m.domain_margin)
            if layout:
                mh.save(layout)
            return mh
        shared = os.path.join("/tmp", f"p2m_bench_{os.getpid() if world == 1 else 'shared'}.p2m")
        mesh = share_layout(rank, world, build_and_keep, pg.P2M.load, shared, dist)
        if world > 1 and rank == 0:  # every replica has loaded it (share_layout's barrier)
            try:
                os.remove(shared)
            except OSError:
                pass
    build_s = time.perf_counter() - t0
    st = mesh.stats()
    q = torch.from_numpy(m.queries).cuda()
    out = out_buffers(torch, n)
    mesh.reserve(n)
    tuned_ms = None
    if args.tuning:
        mesh.tuning = json.loads(args.tuning)
    if not args.no_autotune:
        tuned_ms = mesh.autotune(q, reps=2)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, warmup)):
        mesh.query(q, out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    ms = timed(lambda: mesh.query(q, out=out), steps, stream, flush)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks([ms], dist)[0]
    conc = None
    if flush is None and world == 1:
        conc = concurrent_steps(mesh, q, n, steps, args.pipe_depth)
    tsum = phase_times(mesh, q, out, steps, flush)
    roof = forward_roofline(mesh, q, n, tsum, ms / steps, steps)
    e2e_s, serial_s = pipe_e2e(mesh, m, steps, dist, args.pipe_depth)
    e2e_s, serial_s = max_over_ranks([e2e_s, serial_s], dist)
    res = {"value": replica_throughput(n, steps, world, ms / 1e3), "unit": UNIT,
           "ms_per_step": ms / steps, "steps": steps, "warmup": max(3, warmup),
           "clocks": clk, "roofline": roof,
           "e2e": {"value": replica_throughput(n, steps, world, e2e_s), "unit": UNIT,
                   "h2d_bytes_per_step": 12 * n, "d2h_bytes_per_step": 21 * n,
                   "outputs": "dist, prim_id, closest, prim_type (all of them, 21 B per query)",
                   "api": f"p2m_pipe_submit, {args.pipe_depth} slots (pinned host buffers)",
                   "serial_value": replica_throughput(n, steps, world, serial_s),
                   "serial_api": "p2m_query_host (synchronous per step)"},
           "gpu_launches": kernels_per_step(mesh.tuning, n) * steps,
           "concurrent_steps": conc,
           "run": {"tuning": mesh.tuning, "autotune_ms": tuned_ms, "build_s": round(build_s, 1),
                   "layout_gb": round(st["device_bytes"] / 1e9, 3),
                   "table_entries": st["n_entries"], "max_list": st["max_list"],
                   "build_split_ms": {"cells": st["cells_ms"],
                                      "flooding_and_packing": st["inspect_ms"]},
                   "flooding": mesh.flood_stats(), "cells": mesh.cell_stats()}}
    mesh.close()
    del q, out
    torch.cuda.empty_cache()
    return res


def small_config(pg, idx, args, local):
    """Workloads 0 and 2 (plain forward) as sub-objects of the line."""
    import torch
    m = dg.workload(idx)
    n = m.queries.shape[0]
    flush = None
    steps = args.steps
    if idx == 0:
        # the whole problem fits in L2: rewrite a buffer larger than L2
        # between the timed steps (outside their events), and take more steps
        flush = torch.empty(2 * L2_BYTES // 4, device="cuda")
        steps = max(args.steps, 100)
    r = measure_forward(pg, m, args, local, steps=steps, warmup=args.warmup, flush=flush)
    r["config"] = {"workload": m.name, "n_tris": int(m.tris.shape[0]),
                   "n_verts": int(m.verts.shape[0]), "n_queries": n,
                   "l2": "L2 flushed between steps (a 258 MB buffer rewritten outside the "
                         "events)" if flush is not None else
                         "inputs larger than L2 (layout and queries), no flush"}
    return r


def run_fwd_bwd(pg, args, local):
    """Workload 3: loss = sum w_i d_i on the noisy 7x-subdivided icosphere,
    4M near-surface queries; forward+backward (gradients to the queries and
    to the vertex positions) against the forward alone, same GPU, same
    queries; the backward kernel alone for its roofline."""
    import torch
    m = dg.workload(3, n_queries=args.queries, level=args.level)
    n = m.queries.shape[0]
    t0 = time.perf_counter()
    mesh = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin)
    build_s = time.perf_counter() - t0
    q = torch.from_numpy(m.queries).cuda()
    w = torch.from_numpy(m.weights).cuda()
    mesh.reserve(n)
    tuned = mesh.autotune(q, reps=2) if not args.no_autotune else None
    res = mesh.query(q, closest=True, prim_type=False, save=True)
    gv = torch.zeros(m.verts.shape[0], 3, device="cuda")
    stream = torch.cuda.current_stream()

    def fwd():
        mesh.query(q, out=res)

    def bwd():
        gv.zero_()
        mesh.backward(q, res, w, grad_q=True, grad_verts=gv)

    def fwd_bwd():
        fwd()
        bwd()

    for _ in range(max(3, args.warmup)):
        fwd_bwd()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms_f = timed(fwd, args.steps, stream)
    ms_fb = timed(fwd_bwd, args.steps, stream)
    ms_b = timed(bwd, args.steps, stream)
    clk = clocks.stop()
    # end to end through the autograd API: pinned host queries in, forward,
    # backward, the query gradient, the vertex gradient and the loss out
    qh = torch.from_numpy(m.queries).pin_memory()
    gh = torch.empty(n, 3).pin_memory()
    gvh = torch.empty(m.verts.shape[0], 3).pin_memory()
    lh = torch.empty(()).pin_memory()
    verts_d = torch.from_numpy(m.verts).cuda().requires_grad_(True)

    def e2e_step():
        qd = qh.cuda(non_blocking=True).requires_grad_(True)
        d, _ = pg.distance(qd, verts_d, mesh)
        loss = (w * d).sum()
        loss.backward()
        gh.copy_(qd.grad, non_blocking=True)
        gvh.copy_(verts_d.grad, non_blocking=True)
        lh.copy_(loss.detach(), non_blocking=True)
        verts_d.grad = None

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    peak, src = peaks()
    # backward bytes per query: query 12 + saved (typed id, 2 weights) 12 +
    # closest point and distance 16 + weight 4, grad_q out 12, and three
    # vertex gradients read-modify-written (3 x 12 in, 3 x 12 out) plus the
    # three vertex ids 12
    bb = 12 + 12 + 16 + 4 + 12 + 72 + 12
    bwd_ms = ms_b / args.steps
    line = {"value": n * args.steps / (ms_fb / 1e3), "unit": UNIT,
            "metric": "point-to-mesh forward+backward queries/sec (327,680 tris)",
            "ms_per_step": ms_fb / args.steps, "steps": args.steps,
            "warmup": max(3, args.warmup),
            "forward_only": {"value": n * args.steps / (ms_f / 1e3),
                             "ms_per_step": ms_f / args.steps},
            "backward_only": {"value": n * args.steps / (ms_b / 1e3), "ms_per_step": bwd_ms},
            "fwd_bwd_over_fwd_time": ms_fb / ms_f,
            "fwd_over_fwd_bwd_throughput": ms_f / ms_fb,
            "clocks": clk,
            "roofline": {"bound": "hbm", "kernel": "k_backward", "bytes_per_query": bb,
                         "achieved": bb * n / (bwd_ms / 1e3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": bb * n / (bwd_ms / 1e3) / 1e9 / peak,
                         "traffic": None, "kernel_ms": bwd_ms,
                         "note": "backward step (gradient buffer clear + k_backward) timed "
                                 "alone; bytes of the backward per query at minimal record "
                                 "sizes"},
            "e2e": {"value": n * args.steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": 12 * n,
                    "d2h_bytes_per_step": 12 * n + 12 * int(m.verts.shape[0]) + 4,
                    "api": "pg.distance (torch.autograd.Function) from pinned host queries; "
                           "grad_q, grad_verts and the loss copied back"},
            "gpu_launches": (kernels_per_step(mesh.tuning, n) + 1) * args.steps,
            "config": {"workload": m.name, "n_tris": int(m.tris.shape[0]),
                       "n_queries": n, "loss": "sum w_i d_i, w ~ U(0,1)",
                       "grads": "queries and vertex positions",
                       "l2": "inputs larger than L2 (layout and queries), no flush"},
            "run": {"tuning": mesh.tuning, "autotune_ms": tuned, "build_s": round(build_s, 1)}}
    mesh.close()
    torch.cuda.empty_cache()
    return line


def run_batched(pg, args, local):
    """Workload 4: 64 meshes of uneven size in one persistent launch captured
    in a CUDA graph, against the same queries as 64 plain per-mesh launches
    (each mesh autotuned), with the same four outputs."""
    import torch
    scale = 1.0 if args.queries is None else args.queries / 24e6
    ms = dg.batch_workload(64, query_scale=scale)
    t0 = time.perf_counter()
    meshes = [pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale,
                     domain_margin=m.domain_margin) for m in ms]
    build_s = time.perf_counter() - t0
    qs = [torch.from_numpy(m.queries).cuda() for m in ms]
    total = sum(q.shape[0] for q in qs)
    b = pg.P2MBatch(meshes, qs, closest=True, prim_type=True)
    tuned = b.autotune(reps=2)
    tuned_group = bool(b.tuning["group_by_vertex"])
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    b.run(stream=stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        b.run(stream=stream)
    outs = []
    for mesh, q in zip(meshes, qs):
        mesh.reserve(q.shape[0])
        mesh.autotune(q, reps=1)
        outs.append(mesh.query(q, closest=True, prim_type=True))

    def plain():
        for mesh, q, o in zip(meshes, qs, outs):
            mesh.query(q, out=o)

    cur = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        g.replay()
        plain()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms_b = timed(g.replay, args.steps, cur)
    ms_p = timed(plain, args.steps, cur)
    clk = clocks.stop()
    b.check()
    same = all(torch.equal(o[k], r[k]) for o, r in zip(outs, b.out)
               for k in ("dist", "prim_id", "closest", "prim_type"))
    # end to end: every mesh's queries copied in from one pinned host
    # buffer, the graph replayed, every output copied back
    offs = np.cumsum([0] + [q.shape[0] for q in qs])
    qh = torch.from_numpy(np.concatenate([m.queries for m in ms], 0)).pin_memory()
    hout = {"dist": torch.empty(total).pin_memory(),
            "prim_id": torch.empty(total, dtype=torch.int32).pin_memory(),
            "closest": torch.empty(total, 3).pin_memory(),
            "prim_type": torch.empty(total, dtype=torch.uint8).pin_memory()}

    def e2e_step():
        for k, q in enumerate(qs):
            q.copy_(qh[offs[k]:offs[k + 1]], non_blocking=True)
        g.replay()
        for k, r in enumerate(b.out):
            for key, t in r.items():
                hout[key][offs[k]:offs[k + 1]].copy_(t, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    line = {"metric": "batched point-to-mesh queries/sec (64 meshes)",
            "value": total * args.steps / (ms_b / 1e3), "unit": UNIT,
            "ms_per_step": ms_b / args.steps, "steps": args.steps,
            "warmup": max(3, args.warmup),
            "per_mesh_launches": {"value": total * args.steps / (ms_p / 1e3),
                                  "ms_per_step": ms_p / args.steps},
            "batched_over_plain_speedup": ms_p / ms_b, "identical_to_plain": same,
            "clocks": clk,
            "e2e": {"value": total * args.steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": 12 * total, "d2h_bytes_per_step": 21 * total,
                    "api": "torch copies from one pinned host buffer + the batch's CUDA graph"},
            "gpu_launches": (12 if tuned_group else 6) * args.steps,
            "config": {"workload": "batch64-icosphere-heightfield-1k..500k", "meshes": len(ms),
                       "total_tris": int(sum(m.tris.shape[0] for m in ms)),
                       "total_queries": int(total),
                       "l2": "inputs larger than L2 (64 layouts and 24M queries), no flush"},
            "run": {"tuning": b.tuning, "autotune_ms": tuned, "build_s": round(build_s, 1),
                    "launch": "one CUDA graph: sort, nearest-vertex pass, regroup, "
                              "persistent list kernel, output write" if tuned_group else
                              "one CUDA graph: sort + persistent query kernel"}}
    del g
    b.close()
    for mesh in meshes:
        mesh.close()
    torch.cuda.empty_cache()
    return line


def run_ours(args):
    rank, world, local = dist_env()
    worker = None
    threads = os.cpu_count() or 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.only in (None, "headline"):
        # spawned before the first GPU call: the oracle's tables build while
        # the GPU measures
        worker = OracleWorker(args, threads)
    import torch
    import paper_2308_16084_gb300 as pg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    m = workload(args)
    n = m.queries.shape[0]
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_of(m, args)}
    try:
        if args.only in (None, "headline"):
            h = measure_forward(pg, m, args, local, steps=args.steps, warmup=args.warmup,
                                dist=dist, world=world, layout=args.layout)
            line.update({"value": h["value"], "ms_per_step": h["ms_per_step"],
                         "clocks": h["clocks"], "e2e": h["e2e"],
                         "gpu_launches": h["gpu_launches"], "roofline": h["roofline"],
                         "concurrent_steps": h["concurrent_steps"],
                         "run": dict(h["run"], parallelism="replicas only" if world > 1
                                     else "single GPU")})
        if world == 1:
            if args.only in (None, "cfg0", "cfg2"):
                line["configs"] = {}
                for idx in (0, 2):
                    if args.only in (None, f"cfg{idx}"):
                        line["configs"][str(idx)] = guarded(small_config, pg, idx, args, local)
            if args.only in (None, "fwd_bwd"):
                line["fwd_bwd"] = guarded(run_fwd_bwd, pg, args, local)
            if args.only in (None, "batched"):
                line["batched"] = guarded(run_batched, pg, args, local)
            if args.only is not None and args.only != "headline":
                # a profiling run of one part: that part's figures head the line
                part = line.get(args.only) or line["configs"][args.only[-1]]
                for k in ("value", "ms_per_step", "clocks", "e2e", "gpu_launches", "roofline"):
                    if k in part:
                        line[k] = part[k]
        else:
            line["configs_note"] = ("workloads 0, 2, 3 and 4 are measured at one GPU; "
                                    "replicas run the headline only")
        cpu = None
        if worker is not None:
            try:
                built = worker.wait_built(args.cpu_timeout)
                res = worker.time(args.cpu_sample, args.cpu_bf_sample)
                cpu = cpu_baseline_of(res, built, n)
                line["cpu_bruteforce"] = {
                    "value": res["bf_n"] / res["bf_s"], "unit": UNIT, "cores": res["threads"],
                    "kind": "oracle", "sample": f"the first {res['bf_n']} queries of the "
                    "same sample; FP64 brute force over every vertex, open edge and open face"}
            except Exception as e:  # noqa: BLE001
                cpu = {"error": f"{type(e).__name__}: {e}"[:300]}
        line["cpu_baseline"] = cpu
    finally:
        if worker is not None:
            worker.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_sweep(args):
    """Extra workloads (not the headline): mesh resolution, query box,
    triangle soups, a good and a poor triangulation of one sphere, mixed
    primitives, and the per-list R-tree levels on long-list meshes.  One
    JSON line with one entry per case: build seconds, device-resident
    queries/s (CUDA events, 5 steps after 2 warm-ups, default tuning but for
    the R-tree cases) and work per query."""
    import torch
    import paper_2308_16084_gb300 as pg
    n = args.queries or 4_000_000
    cases = []

    def measure(name, mesh, q, extra):
        out = {"dist": torch.empty(q.shape[0], device="cuda"),
               "prim_id": torch.empty(q.shape[0], dtype=torch.int32, device="cuda"),
               "closest": torch.empty(q.shape[0], 3, device="cuda"),
               "prim_type": torch.empty(q.shape[0], dtype=torch.uint8, device="cuda")}
        mesh.reserve(q.shape[0])
        stream = torch.cuda.current_stream()
        ms = timed(lambda: mesh.query(q, out=out), 2, stream)
        ms = timed(lambda: mesh.query(q, out=out), 5, stream) / 5
        cnt = mesh.counters(q)
        st = mesh.stats()
        cases.append({"case": name, "n_tris": mesh.n_tris, "n_queries": int(q.shape[0]),
                      "queries_per_s": q.shape[0] / (ms / 1e3), "ms": ms,
                      "entries_per_vertex": st["n_entries"] / max(1, mesh.n_verts),
                      "work_per_query": {k: round(v / q.shape[0], 2) for k, v in cnt.items()},
                      **extra})
        print(json.dumps(cases[-1]), file=sys.stderr, flush=True)

    def build(m, segs=None, scale=None):
        t0 = time.perf_counter()
        mesh = pg.P2M(m.verts, m.tris, segs=segs,
                      domain_scale=m.domain_scale if scale is None else scale,
                      domain_margin=m.domain_margin)
        return mesh, time.perf_counter() - t0

    # mesh resolution (workload 1's recipe at coarser levels)
    for lvl in (5, 6, 7):
        m = dg.workload(1, n_queries=n, level=lvl)
        mesh, bs = build(m)
        measure(f"resolution L{lvl}", mesh, torch.from_numpy(m.queries).cuda(),
                {"build_s": round(bs, 1), "queries": "uniform in bbox x1.5"})
    # query box on one mesh whose domain covers the widest box
    m = dg.workload(1, n_queries=16, level=7)
    mesh, bs = build(m, scale=3.2)
    rq = np.random.default_rng(np.random.SeedSequence(dg.ROOT_SEED).spawn(8)[7])
    diag = dg.bbox_diagonal(m.verts)
    tris_f = m.tris.astype(np.int64)
    boxes = [("near 0.01 diag", dg.near_surface(m.verts.astype(np.float64), tris_f, n, 0.01 * diag, rq))]
    for sc in (1.2, 1.5, 3.0):
        boxes.append((f"uniform bbox x{sc}", dg.uniform_in_box(m.verts.astype(np.float64), sc, n, rq)))
    for label, qq in boxes:
        measure(f"query box: {label}", mesh, torch.from_numpy(qq.astype(np.float32)).cuda(),
                {"build_s": round(bs, 1), "domain": "bbox x3.2 + 0.01 diag"})
    # triangle soups (the paper's soup test) and mixed primitives
    for kind in ("watertight", "gapped", "penetrating"):
        m = dg.soup_workload(kind, level=4, n_queries=min(n, 1_000_000))
        mesh, bs = build(m)
        measure(f"soup {kind} (5,120 faces)", mesh, torch.from_numpy(m.queries).cuda(),
                {"build_s": round(bs, 1)})
    # good and poor triangulations of one surface (Table 5 analogue)
    for label, m in zip(("good: noisy icosphere L5", "poor: noisy lat-long sphere 32x320"),
                        dg.triangulation_pair(min(n, 2_000_000))):
        mesh, bs = build(m)
        q_mean, slivers = dg.triangle_quality(m.verts, m.tris)
        measure(f"triangulation {label}", mesh, torch.from_numpy(m.queries).cuda(),
                {"build_s": round(bs, 1), "mean_Q": round(q_mean, 3),
                 "min_angle_below_10deg": round(slivers, 3)})
    m = dg.mixed_workload(mesh_level=6, wire_level=4, n_queries=min(n, 2_000_000))
    mesh, bs = build(m, segs=m.meta["segs"])
    measure("mixed: mesh L6 + wireframe L4", mesh, torch.from_numpy(m.queries).cuda(),
            {"build_s": round(bs, 1), "n_segments": int(m.meta["segs"].shape[0])})
    # per-list R-tree (Table 4 analogue): the same queries scanned with the
    # Region box of every entry (chunked 0), chunk boxes first (1) and
    # super-chunk boxes first (2), on meshes with long lists
    for label, m in rtree_meshes(min(n, 2_000_000)):
        mesh, bs = build(m)
        qd = torch.from_numpy(m.queries).cuda()
        for mode in (0, 1, 2):
            mesh.tuning = {"chunked": mode}
            measure(f"R-tree levels {mode}: {label}", mesh, qd,
                    {"build_s": round(bs, 1), "max_list": int(mesh.stats()["max_list"])})
    line = {"metric": "point-to-mesh queries/sec by workload (sweep)", "unit": UNIT,
            "n_gpus": 1, "data": "synthetic", "dtype": "f32", "higher_is_better": True,
            "sweep": cases}
    print(json.dumps(line), flush=True)
    return 0


def rtree_meshes(n):
    """Meshes with long interception lists for the R-tree comparison: the
    displaced icosphere at level 6 (lists of 99 entries on average, up to
    658) and a gapped soup of an exact, noise-free icosphere at level 3
    (every face shrunk to 80 % about its centroid: the cells of its
    cospherical vertices meet at the centre, so its lists hold most faces).
    Queries: half uniform in the bbox scaled 1.2x, half near the surface."""
    rq = np.random.default_rng(np.random.SeedSequence(dg.ROOT_SEED).spawn(9)[8])
    out = [("displaced icosphere L6", dg.workload(1, n_queries=n, level=6))]
    v, f = dg.icosphere(3)
    tri = v[f]
    c = tri.mean(1, keepdims=True)
    sv = (c + 0.8 * (tri - c)).reshape(-1, 3)
    sf = np.arange(sv.shape[0]).reshape(-1, 3)
    half = n // 2
    q = np.concatenate([dg.uniform_in_box(sv, 1.2, half, rq),
                        dg.near_surface(sv, sf, n - half, 0.01 * dg.bbox_diagonal(sv), rq)], 0)
    out.append(("exact-sphere gapped soup L3",
                dg.Mesh("exact-sphere-gapped-soup-L3", sv.astype(np.float32),
                        sf.astype(np.int32), q.astype(np.float32), 1.25, 0.02, meta={})))
    return out


def run_list_stats(args):
    """Interception-list statistics of the built tables (host build; no GPU
    needed, the certification runs on one when present): per workload the
    vertices, faces, edges and table entries, the average and maximum
    numbers of intercepted edges and faces per vertex (the per-vertex
    columns of the paper's Table 2), list-length percentiles (the histogram
    of Sec. 5.1), vertex inspections per flooded primitive and the share of
    visited vertices that do not intercept, the layout's bytes by part
    (Sec. 5.4), the build time split (Table 3) and the triangle quality of
    Sec. 5.5 (a noisy icosphere and a noisy latitude-longitude sphere stand
    in for Table 5's good and poor triangulations of one surface).  One JSON line per case on stderr, then one line
    with every case on stdout."""
    import paper_2308_16084_gb300 as pg
    cases = [
        ("noisy icosphere L3 (workload 0)", lambda: dg.workload(0, n_queries=10)),
        ("displaced icosphere L6 (workload 1 at level 6)",
         lambda: dg.workload(1, n_queries=10, level=6)),
        ("noisy icosphere L7 (workload 3)", lambda: dg.workload(3, n_queries=10)),
        ("jittered height field 256^2 (workload 2 at 256^2)",
         lambda: dg.workload(2, n_queries=10, grid=256)),
        ("sphere, good triangulation: noisy icosphere L5",
         lambda: dg.triangulation_pair(10)[0]),
        ("sphere, poor triangulation: noisy lat-long 32x320",
         lambda: dg.triangulation_pair(10)[1]),
        ("soup gapped L5", lambda: dg.soup_workload("gapped", level=5, n_queries=10)),
        ("soup penetrating L5", lambda: dg.soup_workload("penetrating", level=5, n_queries=10)),
        ("mesh L6 + wireframe L4", lambda: dg.mixed_workload(6, 4, n_queries=10)),
    ]
    rows = []
    for name, make in cases:
        m = make()
        t0 = time.perf_counter()
        mesh = pg.P2M(m.verts, m.tris, segs=m.meta.get("segs"), domain_scale=m.domain_scale,
                      domain_margin=m.domain_margin)
        build_s = time.perf_counter() - t0
        st = mesh.stats()
        ne = np.zeros(mesh.n_verts, np.int64)
        nf = np.zeros(mesh.n_verts, np.int64)
        for v in range(mesh.n_verts):
            t, _, _ = mesh.interception_list(v)
            ne[v] = int((t == 1).sum())
            nf[v] = int((t == 2).sum())
        ln = ne + nf
        fs = mesh.flood_stats()
        # layout bytes by part (the record sizes of the device layout; the
        # seed grids and the query scratch come on top, on the device only)
        chunks = (ln + 7) // 8
        supers = (chunks + 7) // 8
        nvp = mesh.n_verts + 1
        parts = {
            "kd_tree": 48 * (st["kd_leaves"] - 1) + 16 * mesh.n_verts,
            "voronoi_neighbours": 4 * nvp + 20 * st["neighbour_pairs"],
            "interception_entries": 16 * int(st["n_entries"]) + 4 * nvp,
            "r_tree_boxes": 16 * int(chunks.sum() + supers.sum()) + 8 * nvp,
            "geometry": 40 * mesh.n_edges + 64 * mesh.n_tris,
        }
        q_mean, slivers = dg.triangle_quality(m.verts, m.tris) if m.tris.shape[0] else (0, 0)
        rows.append({
            "case": name, "n_verts": mesh.n_verts, "n_tris": mesh.n_tris,
            "triangle_quality": {"mean_Q": round(q_mean, 3),
                                 "min_angle_below_10deg": round(slivers, 3)},
            "n_edges": mesh.n_edges, "entries": int(st["n_entries"]),
            "edges_per_vertex": {"avg": round(float(ne.mean()), 2), "max": int(ne.max())},
            "faces_per_vertex": {"avg": round(float(nf.mean()), 2), "max": int(nf.max())},
            "list_length": {"avg": round(float(ln.mean()), 2),
                            **{f"p{q}": int(np.percentile(ln, q)) for q in (10, 50, 90, 99)},
                            "max": int(ln.max())},
            "inspections_per_primitive": round(st["inspections"] / max(1, sum(fs.values())), 2),
            # share of the vertices the flooding visited that do not intercept
            # (the paper reports about 85 %, Sec. 6)
            "visited_rejected": round(1.0 - st["n_entries"] / max(1, st["inspections"]), 3),
            "layout_mb": {k: round(v / 1e6, 2) for k, v in parts.items()},
            "build_s": round(build_s, 2), "cells_ms": int(st["cells_ms"]),
            "flooding_and_packing_ms": int(st["inspect_ms"]),
        })
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"list_stats": rows}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.list_stats:
        return run_list_stats(args)
    if args.sweep:
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
