"""The multi-process host logic of bench.py on CPU: world_size-2 gloo ranks (no GPU).

Each rank runs its own replica catalog; the timed region is the slowest rank's; the value
is every rank's units over that time."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    assert bench.dist_env() == (ws, rank, rank)
    ms = 2.0 + 3.0 * rank          # rank 1 is the slow one
    got = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.whole_job_rate(ws, 1000, got * 1e-3)
    q.put((rank, got, rate, bench.replica_seed(2, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_distinct_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, s0), (r1, ms1, v1, s1) = out
    assert ms0 == ms1 == 5.0
    assert v0 == v1 == pytest.approx(2 * 1000 / 5e-3)
    assert s0 == 2 and s1 != s0


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(1, 10, 2.0) == 5.0
    assert bench.replica_seed(7, 0) == 7
