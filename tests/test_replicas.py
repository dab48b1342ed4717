"""Multi-GPU is replicas only (the render shards across views, no data-path
exchange): each rank renders its own frames of the sweep and the job's time
is the slowest rank's. The host-side logic of that path, run as two gloo
ranks on the CPU."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q) -> None:
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        frames = bench.frames_for_rank(rank, 40)
        slowest = bench.max_over_ranks(10.0 * (rank + 1))
        q.put((rank, frames, slowest))
    finally:
        dist.destroy_process_group()


def test_two_replicas_share_the_sweep_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict()
    for _ in procs:
        rank, frames, slowest = q.get(timeout=120)
        out[rank] = (frames, slowest)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    f0, f1 = out[0][0], out[1][0]
    assert len(f0) == len(f1) == 40
    assert not set(f0) & set(f1)  # disjoint frames
    assert all(0 <= k < 300 for k in f0 + f1)
    assert out[0][1] == out[1][1] == 20.0  # max over ranks


def test_single_process_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.frames_for_rank(0, 3) == [0, 7, 14]
