"""The N > 1 benchmark path on CPU: independent replicas, combined with gloo (world size 2).

Replicas exchange no solver data; the only collective is the combination of timing figures
(slowest rank's time, sum of all ranks' work units), checked here without a GPU.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as td
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.combine_ranks(10.0 + 5.0 * rank, 100.0 * (rank + 1), device="cpu")
    out[rank] = (t, u)
    td.destroy_process_group()


def test_combine_ranks_max_time_sum_units():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r] == (15.0, 300.0)


def test_reference_arm_other_ranks_do_nothing():
    import bench
    args = type("A", (), {"steps": 1, "warmup": 0})()
    assert bench.run_reference(args, ws=2, rank=1) is None
