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


def test_roofline_of_the_dominant_kernel():
    sys.path.insert(0, ROOT)
    import bench
    tr = {"median": {"dram_bytes_per_launch": 1.2e7, "units_first_launch": 1222,
                     "warp_inst_per_unit": 7.0e4, "kernel_source_sha256": "abc"},
          "prepass": {"dram_bytes_per_launch": 8.1e8, "kernel_source_sha256": "abc"}}
    med = {"ms_per_run": 0.5, "launches_per_run": 17.0, "units_per_run": 2432,
           "algorithmic_bytes_per_run": 7.0e7}
    r = bench.dominant_roofline("median", med, tr, "abc", 6700.0, "of measured", 152, 2070.0)
    # algorithmic bytes of the work handed out, per average launch, over the HBM peak
    per_launch_s = 0.5e-3 / 17
    assert r["bound"] == "hbm" and r["peak"] == 6700.0
    assert r["achieved"] == pytest.approx(7.0e7 / 17 / per_launch_s / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] == pytest.approx(1.2e7 * (2432 / 17) / 1222)
    # the issue rate beside it: warp instructions over one per scheduler per clock
    iv = r["issue_view"]
    assert iv["peak"] == pytest.approx(152 * 4 * 2.07)
    assert iv["achieved"] == pytest.approx(7.0e4 * 2432 / 17 / per_launch_s / 1e9)
    assert iv["frac"] == pytest.approx(iv["achieved"] / iv["peak"])
    # a capture of other sources: no traffic, and the instruction counts flagged
    stale = bench.dominant_roofline("median", med, tr, "new", 6700.0, "of measured", 152, 2070.0)
    assert stale["bound"] == "hbm" and stale["traffic"] is None
    assert "stale" in stale["issue_view"]["instructions_from"]
    pre = {"ms_per_run": 0.5, "launches_per_run": 1.0, "units_per_run": None,
           "algorithmic_bytes_per_run": 7.6e8}
    p = bench.dominant_roofline("prepass", pre, tr, "abc", 6700.0, "of measured", 152, 2070.0)
    assert p["bound"] == "hbm" and p["achieved"] == pytest.approx(7.6e8 / 0.5e-3 / 1e9)
    assert p["traffic"] == 8.1e8 and p["frac"] == pytest.approx(p["achieved"] / 6700.0)


def test_loop_units_follow_the_estimator_lists():
    sys.path.insert(0, ROOT)
    import bench
    work = {"changed": 10, "within1": 20, "within2": 30, "tiles": 15}
    assert [bench.loop_units(k, work, 2) for k in ("sort", "median", "prefix", "mean")] == [
        10, 15, 20, 30]
    assert [bench.loop_units(k, work, 0) for k in ("prefix", "mean")] == [10, 20]
    assert bench.loop_units("median", work, 1) == 15 and bench.loop_units("snr", work, 2) is None
    assert bench.unit_bytes("median", 1024, 2) == 28 * 1024
