"""The multi-rank host logic of the benchmark on CPU (gloo, world size 2):
each rank solves its own designs (disjoint seeds, no data exchange) and the
whole-job throughput divides all ranks' units by the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        seeds = bench.design_seeds(100, rank, 4)
        local_ms = 100.0 * (rank + 1)  # rank 1 is the slow one
        value, t = bench.job_throughput(local_ms, 4 * 10, dist, "cpu")
        out[rank] = (seeds, value, t)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_designs_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    s0, v0, t0 = res[0]
    s1, v1, t1 = res[1]
    assert not set(s0) & set(s1)                  # disjoint designs
    assert t0 == t1 == 200.0                       # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(2 * 40 / 0.2)  # all units / max time


def test_single_process_throughput():
    v, t = bench.job_throughput(50.0, 10)
    assert t == 50.0 and v == pytest.approx(200.0)


def test_design_seeds_stay_disjoint_at_the_default_batch():
    """Every rank of an 8-GPU run solves its own 1024 designs: no seed repeats
    across ranks (the per-rank stride exceeds the batch)."""
    seen = set()
    for r in range(8):
        s = bench.design_seeds(2605_04735 + 1, r, 1024)
        assert len(set(s)) == 1024 and not seen & set(s)
        seen |= set(s)
    assert bench.design_seeds(2605_04735 + 1, 0, 3) == [2605_04736, 2605_04737, 2605_04738]
