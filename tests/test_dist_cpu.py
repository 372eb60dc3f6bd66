"""Multi-rank benchmark logic on CPU (gloo, world size 2; no GPU).

Frames are independent, so the benchmark shards them across ranks with no
collective on the data path: each rank times its own frames and the job's
time is the slowest rank's.  These tests run two gloo ranks on 127.0.0.1 and
check the reduction and the whole-job throughput arithmetic of bench.py."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, _ = bench._dist()
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        slowest = bench.max_over_ranks(ms)
        value = bench.weak_scaling_value(1_000_000, ws, slowest / 1e3)
        out.put((r, ws, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_the_slowest_and_count_all_frames():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for _, ws, slowest, value in res:
        assert ws == 2
        assert slowest == 15.0
        assert value == pytest.approx(2_000_000 / 0.015)


def test_single_process_is_unchanged():
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.weak_scaling_value(10, 1, 2.0) == 5.0
