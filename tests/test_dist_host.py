"""The multi-rank host logic of bench.py on CPU: two gloo ranks (one process each, the
way torchrun starts replicas), each with its own step time; every rank must see the
slowest time, and the job's throughput counts both ranks' samples over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    ws, r, _ = bench.dist_env()
    dist = bench.dist_init(ws, backend="gloo")
    bench.barrier(dist, torch)
    ms = 3.0 + 2.0 * r                     # rank 1 is the slow one
    ms_max = bench.max_over_ranks(dist, torch, ms)
    q.put((r, ms_max, bench.aggregate_gsas(ws, ms_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_and_count_both():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    import bench
    for r, ms_max, gsas in res:
        assert ms_max == 5.0
        assert gsas == pytest.approx(2 * bench.NSAMP / 5e-3 / 1e9)
