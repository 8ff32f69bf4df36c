"""The N>1 bookkeeping of bench.py on CPU: two gloo ranks, weak scaling, job time =
max over ranks, throughput counts both ranks' elements."""
import os
import socket

import torch
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1605_01020_gb300.dist import max_over_ranks, weak_scaling_throughput
    ms_local = 100.0 + 50.0 * rank            # rank 1 is slower
    value, ms = weak_scaling_throughput(4096, 5, ms_local)
    a, b = max_over_ranks([rank, -rank])
    out[rank] = (value, ms, a, b)
    torch.distributed.destroy_process_group()


def test_weak_scaling_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        value, ms, a, b = out[r]
        assert ms == 150.0
        assert abs(value - 4096 * 5 * 2 / 0.150) < 1e-6
        assert a == 1.0 and b == 0.0
