"""The benchmark's multi-process plumbing (replicas: barrier plus max / sum of
the timings, no data-path collective) on two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port), "LOCAL_RANK": str(rank)})
    import bench
    r, w = bench.init_dist(backend="gloo")
    assert (r, w) == (rank, world)
    bench.barrier(w)
    mx = bench.allreduce_max(10.0 * (rank + 1), w)
    sm = bench.allreduce_sum(rank + 1, w)
    out.put((rank, mx, sm))
    bench._PG.destroy_process_group()


def test_two_gloo_ranks_reduce_timings():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 20.0, 3.0), (1, 20.0, 3.0)]


def test_single_process_needs_no_group():
    import bench
    assert bench.init_dist() == (0, 1) or os.environ.get("WORLD_SIZE") not in (None, "1")
    assert bench.allreduce_max(3.5, 1) == 3.5
