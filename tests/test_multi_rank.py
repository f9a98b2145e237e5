"""The multi-GPU path is replicas over frames (no data-path collective):
each rank renders its own frames of the trajectory and the reported value is
the units of all ranks over the slowest rank's time. The host logic runs here
as world_size-2 gloo ranks on CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        frames = bench.shard_frames(rank, world, 10)
        units = float(len(frames) * 1000 + rank)           # rank-specific work
        seconds = 1.0 + rank                                # rank 1 is slower
        value = bench.whole_job_throughput(units, seconds, world, device="cpu")
        mx = bench._max_over_ranks(seconds, world, device="cpu")
        out[rank] = (frames, value, mx)
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_whole_job_value():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    f0, v0, m0 = out[0]
    f1, v1, m1 = out[1]
    assert set(f0).isdisjoint(f1) and len(f0) == len(f1) == 10
    assert sorted(f0 + f1) == list(range(20))
    # sum of units over the slowest rank's time, identical on both ranks
    assert v0 == v1 == pytest.approx((10000 + 10001) / 2.0)
    assert m0 == m1 == 2.0


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.shard_frames(0, 1, 5) == [0, 1, 2, 3, 4]
    assert bench.whole_job_throughput(10.0, 2.0, 1) == 5.0
