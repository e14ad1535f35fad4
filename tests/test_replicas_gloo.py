"""The bench's multi-GPU form is replicas (one table per rank, no data
exchange): only the job's timing crosses ranks.  Two gloo ranks on the CPU
check that every rank gets the slowest rank's time and the job's throughput
counts all ranks' bytes."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank
    q.put((rank,) + bench.replica_throughput(local_ms, step_bytes=10**9, steps=4, world=world, device="cpu"))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, ms, gbs in got:
        assert ms == 150.0
        assert abs(gbs - 2 * 4 * 1e9 / 0.150 / 1e9) < 1e-9


def test_single_rank_is_unchanged():
    ms, gbs = bench.replica_throughput(80.0, step_bytes=2 * 10**9, steps=5, world=1, device="cpu")
    assert ms == 80.0 and abs(gbs - 125.0) < 1e-9
