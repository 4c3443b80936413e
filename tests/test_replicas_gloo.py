"""The multi-GPU bench runs independent replicas (no data-path collective): the
whole-job value is all ranks' units over the slowest rank's time. Checked with
two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r timed (100 + 50 r) ms for 3 steps of 1e9 contributions
    t = bench.max_over_ranks(100.0 + 50.0 * rank, dist, "cpu")
    v = bench.replica_value(world, 1e9, 3, t)
    dist.barrier()
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_replicas_value_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 150.0
        assert v == pytest.approx(2 * 1e9 * 3 / 0.150)


def test_single_rank_value():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.replica_value(1, 2.4576e10, 5, 2200.0) == pytest.approx(5.5855e10, rel=1e-4)
