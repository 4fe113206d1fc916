#!/usr/bin/env python3
"""Benchmark of the point-to-mesh query stage on GB300.

One step = one pass of the whole query path (Morton bucket sort, KD-tree
nearest vertex, interception-list scan with Region-box filter, edge/face
tests, minimum, outputs in caller order) over the 10M uniform queries of the
1.3M-triangle displaced icosphere.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 oracle (the plain brute-force definition of
the distance, all host cores) on a bounded sample of the same workload.
For N > 1 (torchrun) every rank runs an independent replica (the query path
has no exchange step): value = all ranks' queries / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import datagen as dg  # noqa: E402

METRIC = "point-to-mesh queries/sec (1.3M tris)"
UNIT = "queries/s"
WORKLOAD = 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=1024,
                    help="queries of the bounded CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--level", type=int, default=None, help="smaller mesh (profiling only)")
    ap.add_argument("--queries", type=int, default=None, help="fewer queries (profiling only)")
    ap.add_argument("--workload", type=int, default=1, choices=[1, 3, 4],
                    help="1: forward queries (default); 3: forward+backward; 4: 64-mesh batch")
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
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args):
    return dg.workload(WORKLOAD, n_queries=args.queries, level=args.level)


def timed(fn, steps, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_fwd_bwd(args):
    """Workload 3: loss = sum w_i d_i on the noisy 7x-subdivided icosphere,
    4M near-surface queries; forward+backward (grad to the queries and to the
    vertex positions) against the forward alone, same GPU, same queries."""
    import torch
    import paper_2308_16084_gb300 as pg
    m = dg.workload(3, n_queries=args.queries, level=args.level)
    n = m.queries.shape[0]
    t0 = time.perf_counter()
    mesh = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin)
    build_s = time.perf_counter() - t0
    q = torch.from_numpy(m.queries).cuda()
    w = torch.from_numpy(m.weights).cuda()
    mesh.reserve(n)
    mesh.autotune(q, reps=2)
    res = mesh.query(q, closest=True, prim_type=False, save=True)
    gv = torch.zeros(m.verts.shape[0], 3, device="cuda")
    stream = torch.cuda.current_stream()

    def fwd():
        mesh.query(q, out=res)

    def fwd_bwd():
        mesh.query(q, out=res)
        gv.zero_()
        mesh.backward(q, res, w, grad_q=True, grad_verts=gv)

    for _ in range(max(3, args.warmup)):
        fwd_bwd()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.3)
    ms_f = timed(fwd, args.steps, stream)
    ms_fb = timed(fwd_bwd, args.steps, stream)
    clk = clocks.stop()
    # end to end through the autograd API from pinned host memory
    qh = torch.from_numpy(m.queries).pin_memory()
    vh = torch.from_numpy(m.verts).pin_memory()
    gh = torch.empty(n, 3).pin_memory()
    verts_d = vh.cuda().requires_grad_(True)

    def e2e_step():
        qd = qh.cuda(non_blocking=True).requires_grad_(True)
        d, _ = pg.distance(qd, verts_d, mesh)
        (w * d).sum().backward()
        gh.copy_(qd.grad, non_blocking=True)
        verts_d.grad = None

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    v_fb = n * args.steps / (ms_fb / 1e3)
    v_f = n * args.steps / (ms_f / 1e3)
    line = {"metric": "point-to-mesh fwd+bwd queries/sec (327,680 tris)", "value": v_fb,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_fb / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": m.name, "n_tris": int(m.tris.shape[0]),
                       "n_queries_per_gpu": n, "loss": "sum w_i d_i, w ~ U(0,1)",
                       "grads": "queries and vertex positions", "tuning": mesh.tuning,
                       "build_s": round(build_s, 1),
                       "l2": "inputs larger than L2 (layout + 4M queries)"},
            "forward_only": {"value": v_f, "ms_per_step": ms_f / args.steps},
            "fwd_bwd_over_fwd_time": ms_fb / ms_f, "clocks": clk,
            "e2e": {"value": n * args.steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": 12 * n, "d2h_bytes_per_step": 12 * n},
            "gpu_launches": (kernels_per_step(mesh.tuning) + 1) * args.steps,
            "cpu_baseline": None}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args):
    """Workload 4: 64 meshes of uneven size in one persistent launch captured
    in a CUDA graph, against the same queries as 64 plain per-mesh launches."""
    import torch
    import paper_2308_16084_gb300 as pg
    scale = 1.0 if args.queries is None else args.queries / 24e6
    ms = dg.batch_workload(64, query_scale=scale)
    t0 = time.perf_counter()
    meshes = [pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale,
                     domain_margin=m.domain_margin) for m in ms]
    build_s = time.perf_counter() - t0
    qs = [torch.from_numpy(m.queries).cuda() for m in ms]
    total = sum(q.shape[0] for q in qs)
    b = pg.P2MBatch(meshes, qs)
    tuned = b.autotune(reps=2)
    # count, 3 scan kernels, scatter; then either the persistent query kernel
    # or nn pass, 3 scan kernels, vertex scatter, persistent list, output write
    tuned_group = bool(b.tuning["group_by_vertex"])
    stream = torch.cuda.Stream()
    b.run(stream=stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        b.run(stream=stream)
    outs = []
    for mesh, q in zip(meshes, qs):
        mesh.reserve(q.shape[0])
        mesh.autotune(q, reps=1)
        outs.append(mesh.query(q, closest=False, prim_type=False))

    def plain():
        for mesh, q, o in zip(meshes, qs, outs):
            mesh.query(q, out=o)

    cur = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        g.replay()
        plain()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.3)
    ms_b = timed(g.replay, args.steps, cur)
    ms_p = timed(plain, args.steps, cur)
    clk = clocks.stop()
    b.check()
    same = all(torch.equal(o["dist"], r["dist"]) for o, r in zip(outs, b.out))
    line = {"metric": "batched point-to-mesh queries/sec (64 meshes)",
            "value": total * args.steps / (ms_b / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batch64-icosphere-heightfield-1k..500k", "meshes": len(ms),
                       "total_tris": int(sum(m.tris.shape[0] for m in ms)),
                       "total_queries": int(total), "tuning": b.tuning,
                       "autotune_ms": tuned, "build_s": round(build_s, 1),
                       "launch": "one CUDA graph: sort, nearest-vertex pass, regroup, "
                                 "persistent list kernel, output write" if tuned_group else
                                 "one CUDA graph: sort + persistent query kernel"},
            "per_mesh_launches": {"value": total * args.steps / (ms_p / 1e3),
                                  "ms_per_step": ms_p / args.steps},
            "batched_over_plain_speedup": ms_p / ms_b, "identical_to_plain": same,
            "clocks": clk, "gpu_launches": (12 if tuned_group else 6) * args.steps,
            "cpu_baseline": None}
    print(json.dumps(line), flush=True)
    return 0


def config_of(m, args, extra=None):
    c = {"workload": m.name, "mesh": "icosphere subdivided 8x, radial displacement 0.2",
         "n_tris": int(m.tris.shape[0]), "n_verts": int(m.verts.shape[0]),
         "n_queries_per_gpu": int(m.queries.shape[0]),
         "query_distribution": "uniform in bbox scaled 1.5x",
         "domain": f"bbox x{m.domain_scale} + {m.domain_margin} diag"}
    if args.level is not None or args.queries is not None:
        c["reduced"] = True
    if extra:
        c.update(extra)
    return c


# ----------------------------------------------------------------- oracle arm

def oracle_sample(m, k):
    idx = np.linspace(0, m.queries.shape[0] - 1, k).astype(np.int64)
    return idx


def time_oracle(m, n_sample, threads):
    import oracle
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False, threads=threads)
    q = m.queries[oracle_sample(m, n_sample)]
    t0 = time.perf_counter()
    o.bruteforce(q, threads=threads)
    return time.perf_counter() - t0, o


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    m = workload(args)
    threads = os.cpu_count() or 1
    import oracle
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False, threads=threads)
    per = max(16, args.cpu_sample // 8)
    idx = oracle_sample(m, per * (args.steps + args.warmup))
    for s in range(args.warmup):
        o.bruteforce(m.queries[idx[s * per:(s + 1) * per]], threads=threads)
    t0 = time.perf_counter()
    for s in range(args.warmup, args.warmup + args.steps):
        o.bruteforce(m.queries[idx[s * per:(s + 1) * per]], threads=threads)
    dt = time.perf_counter() - t0
    v = per * args.steps / dt
    sample = (f"{per} queries per step, evenly strided over the {m.queries.shape[0]} queries; "
              "FP64 brute force over all vertices, open edges and open faces")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "hardware": "host cores only: rank 0 runs the oracle, the GPUs stay idle",
            "config": config_of(m, args, {"parallelism": f"{threads} host threads"}),
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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


def kernels_per_step(tuning):
    sort = 5 if tuning["sort_bits"] > 0 else 1  # count, 3 scan kernels, scatter
    if tuning.get("group_by_vertex") and not tuning.get("warp_cooperative"):
        return sort + 7  # nn pass, 3 scan kernels, vertex scatter, list pass, output write
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


def run_ours(args):
    import torch
    import paper_2308_16084_gb300 as pg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    m = workload(args)
    n = m.queries.shape[0]

    # build once (rank 0), share the layout file with the other replicas
    t0 = time.perf_counter()
    layout = os.path.join("/tmp", f"p2m_bench_{os.getpid() if world == 1 else 'shared'}.p2m")
    if args.layout and os.path.exists(args.layout):
        mesh = pg.P2M.load(args.layout)
    else:
        def build_and_keep():
            mh = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale,
                        domain_margin=m.domain_margin)
            if args.layout:
                mh.save(args.layout)
            return mh
        mesh = share_layout(rank, world, build_and_keep, pg.P2M.load, layout, dist)
    build_s = time.perf_counter() - t0
    st = mesh.stats()

    q = torch.from_numpy(m.queries).cuda()
    out = {"dist": torch.empty(n, device="cuda"),
           "prim_id": torch.empty(n, dtype=torch.int32, device="cuda"),
           "closest": torch.empty(n, 3, device="cuda"),
           "prim_type": torch.empty(n, dtype=torch.uint8, device="cuda")}
    mesh.reserve(n)
    tuned_ms = None
    if args.tuning:
        mesh.tuning = json.loads(args.tuning)
    if not args.no_autotune:
        tuned_ms = mesh.autotune(q, reps=2)
    stream = torch.cuda.current_stream()

    for _ in range(max(3, args.warmup)):
        mesh.query(q, out=out)
    torch.cuda.synchronize()

    # device-resident timed region
    mesh.set_timing(True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        mesh.query(q, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    tsum = mesh.timing_summary()
    mesh.set_timing(False)
    ms = max_over_ranks([ms], dist)[0]
    value = replica_throughput(n, args.steps, world, ms / 1e3)

    # end to end through the host APIs: pinned host buffers, every step copies
    # its queries in and its distances and ids out inside the timed region.
    # Serial: p2m_query_host (copy in, query, copy out, synchronise).
    # Pipelined: p2m_pipe_submit on two slots, so one step's copies overlap
    # the other step's kernels; the clock stops after the last step's results
    # are in host memory.
    qh = torch.from_numpy(m.queries).pin_memory()
    outs_h = [(torch.empty(n, dtype=torch.float32).pin_memory(),
               torch.empty(n, dtype=torch.int32).pin_memory()) for _ in range(2)]
    for _ in range(2):
        mesh.query_host(qh, *outs_h[0])
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mesh.query_host(qh, *outs_h[0])
    serial_s = time.perf_counter() - t0
    pipe = mesh.pipeline(n, depth=2)
    for k in range(2):
        pipe.submit(qh, *outs_h[k])
    pipe.wait()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        pipe.submit(qh, *outs_h[k % 2])
    pipe.wait()
    e2e_s = time.perf_counter() - t0
    pipe.close()
    e2e_s, serial_s = max_over_ranks([e2e_s, serial_s], dist)
    e2e = {"value": replica_throughput(n, args.steps, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": 12 * n, "d2h_bytes_per_step": 8 * n,
           "api": "p2m_pipe_submit, 2 slots (pinned host buffers)",
           "serial_value": replica_throughput(n, args.steps, world, serial_s),
           "serial_api": "p2m_query_host (synchronous per step)"}

    # roofline of the dominant kernel, timed live over the timed region
    cnt = mesh.counters(q)
    nn_b, list_b, out_b = phase_bytes(cnt, n)
    calls = max(1, tsum["calls"])
    grouped = tsum["nn_ms"] > 0
    phases = {"sort_ms": tsum["sort_ms"] / calls, "nn_pass_ms": tsum["nn_ms"] / calls,
              "regroup_ms": tsum["regroup_ms"] / calls, "list_pass_ms": tsum["list_ms"] / calls,
              "output_ms": tsum["output_ms"] / calls}
    if grouped:
        cand = [("k_nn_pass", phases["nn_pass_ms"], nn_b),
                ("k_list_pass", phases["list_pass_ms"], list_b),
                ("k_unpack", phases["output_ms"], out_b)]
    else:
        cand = [("k_query", phases["list_pass_ms"], nn_b + list_b - 32 + 21)]
    kname, kms, kbytes = max(cand, key=lambda c: c[1])
    peak, src = peaks()
    achieved = kbytes * n / (kms / 1e3) / 1e9
    traffic = measured_traffic(kname, n)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured"
            else "fallback 6.8 TB/s",
            "kernel": kname, "kernel_ms": kms, "bytes_per_query": kbytes,
            "note": "achieved counts every list and geometry byte each query reads; after "
                    "the regrouping by nearest vertex the lanes of a warp share one list, so "
                    "most of those reads hit L1/L2 and frac can exceed 1; traffic is the "
                    "DRAM bytes per launch from ncu",
            "phases": phases, "bytes_per_query_by_kernel": {"k_nn_pass": nn_b, "k_list_pass": list_b,
                                          "k_unpack": out_b},
            "work_per_query": {k: v / n for k, v in cnt.items()}}
    if traffic:
        # the DRAM side of the same launch: its ncu DRAM bytes over its live
        # duration, against the same peak
        roof["dram_achieved"] = traffic / (kms / 1e3) / 1e9
        roof["dram_frac"] = roof["dram_achieved"] / peak

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        dt, _ = time_oracle(m, args.cpu_sample, threads)
        cpu = {"value": args.cpu_sample / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{args.cpu_sample} of the {n} queries (evenly strided), FP64 brute "
                         "force over all vertices, open edges and open faces"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": config_of(m, args, {
                "parallelism": "replicas only" if world > 1 else "single GPU",
                "l2": f"inputs larger than L2: layout {st['device_bytes'] / 1e9:.2f} GB + "
                      f"queries {12 * n / 1e6:.0f} MB per step",
                "tuning": mesh.tuning, "autotune_ms": tuned_ms, "build_s": round(build_s, 1),
                "table_entries": st["n_entries"], "max_list": st["max_list"],
                "build_split_ms": {"cells": st["cells_ms"],
                                   "flooding_and_packing": st["inspect_ms"]},
                "flooding": mesh.flood_stats()}),
            "clocks": clk, "e2e": e2e, "gpu_launches": kernels_per_step(mesh.tuning) * args.steps,
            "roofline": roof, "cpu_baseline": cpu}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0 and world > 1:
        try:
            os.remove(layout)
        except OSError:
            pass
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
    if args.workload == 3:
        return run_fwd_bwd(args)
    if args.workload == 4:
        return run_batched(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
