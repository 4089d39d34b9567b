"""The N > 1 host path of bench.py on two gloo ranks (CPU): independent points per rank,
barrier, max over ranks, whole-job throughput, and the reference arm running on rank 0 only."""
from __future__ import annotations

import os
import socket
import sys
from pathlib import Path

import pytest
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parents[1]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, str(ROOT))
    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    # rank r took (r + 1) * 10 ms for 4 steps of 1000 units each
    ms, value = bench.whole_job(w, 10.0 * (rank + 1), 4, 1000)
    called = []

    class _Args:   # the reference arm must not run its oracle pool on rank > 0
        steps, warmup, ref_seconds = 1, 0, 0.01
    if rank != 0:
        orig = bench.OraclePool
        bench.OraclePool = lambda: called.append(1)
        bench.run_reference(_Args, w, r)
        bench.OraclePool = orig
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    out.put((rank, ms, value, bench.point_seed(rank), len(called)))


def test_two_gloo_ranks_whole_job_and_independent_points():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    assert codes == [0, 0], codes
    res = sorted(q.get(timeout=5) for _ in range(world))
    # every rank sees the slowest rank's time; the job processed both ranks' units
    for rank, ms, value, seed, called in res:
        assert ms == pytest.approx(20.0 / 4)
        assert value == pytest.approx(2 * 1000 / (5.0e-3))
        assert called == 0
    # each rank marginalises its own point
    assert len({r[3] for r in res}) == world
