"""The multi-GPU mode of bench.py is replicas only (the query path has no
exchange step): rank 0 builds and shares the layout file, every rank runs
the whole workload, the slowest rank's time sets the job's rate.  These
checks run that coordination as two gloo processes on the CPU."""
import os
import socket
import tempfile

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, tmp, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import datagen as dg
    import paper_2308_16084_gb300 as pg
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        # the slowest rank sets each time; the rate counts every rank's units
        times = bench.max_over_ranks([1.0 + rank, 5.0 - rank], dist)
        rate = bench.replica_throughput(1000, 4, world, times[0])
        # rank 0 builds, the others load its layout file
        m = dg.workload(0, n_queries=10, level=1)
        path = os.path.join(tmp, "layout.p2m")
        mesh = bench.share_layout(
            rank, world,
            lambda: pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale,
                           domain_margin=m.domain_margin, device_assist=False),
            pg.P2M.load, path, dist)
        st = mesh.stats()
        q.put((rank, times, rate, st["n_entries"], mesh.edges().tolist()))
    finally:
        dist.destroy_process_group()


def test_replicas_share_layout_and_take_the_slowest_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with tempfile.TemporaryDirectory() as tmp:
        procs = [ctx.Process(target=_worker, args=(r, world, port, tmp, q)) for r in range(world)]
        for p in procs:
            p.start()
        out = [q.get(timeout=180) for _ in range(world)]
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
    out.sort()
    for rank, times, rate, n_entries, edges in out:
        assert times == [2.0, 5.0]
        assert rate == pytest.approx(1000 * 4 * world / 2.0)
    assert out[0][3] == out[1][3] > 0
    assert out[0][4] == out[1][4]
