"""The N > 1 path of bench.py on CPU: two gloo ranks (spawned processes,
rendezvous on 127.0.0.1). Every rank decomposes its own matrix (replicas, no
collective on the data path); the job's step time is the slowest rank's,
taken by an all-reduce MAX, and the whole-job rate is world / that time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    w, r, local = bench.dist_setup()
    ms = [12.5, 20.0, 16.0, 9.0][r]            # per-rank step times
    slow = bench.max_over_ranks(ms, w, "cpu")
    q.put((r, w, local, slow, bench.aggregate_rate(slow, w)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_slowest_rank_sets_the_job_rate(world):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = max([12.5, 20.0, 16.0, 9.0][:world])
    for r, w, local, slow, rate in out:
        assert w == world and local == r
        assert slow == want
        assert rate == pytest.approx(world * 1000.0 / want)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.aggregate_rate(25.0, 1) == pytest.approx(40.0)
