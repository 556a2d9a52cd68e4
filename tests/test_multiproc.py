"""The benchmark's N > 1 host path on CPU: two ranks over gloo (127.0.0.1)
run independent replicas, meet at barriers, and report the slowest rank's
time and the whole-job aggregate (no data-path collective)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    out[rank] = (ms, bench.aggregate(1000, ms, world))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_rank_gloo_max_and_aggregate():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] == pytest.approx(2 * 1000 / 0.015)
