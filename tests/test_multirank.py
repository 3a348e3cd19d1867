"""The multi-rank path of bench.py on the CPU: two gloo ranks combine their figures the way the
bench does on N GPUs (slowest rank's time, total feasible count).  Instances are independent,
so this reduction is the run's only collective."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms, counts, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        t, c = bench.combine_ranks(dist, ms[rank], counts[rank], "cpu")
        out[rank] = (t, c)
    finally:
        dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks():
    world = 2
    ms = [812.5, 799.25]
    counts = [3421, 3398]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), ms, counts, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (max(ms), sum(counts))
