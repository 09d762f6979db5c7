"""The multi-GPU path of bench.py on CPU: two gloo ranks, each with its own
replica (different work and timings), reduce to the slowest rank's time and
the sum of the work; one rank is a no-op."""
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


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        mx, sm = bench.reduce_over_ranks([10.0 + rank, 3.0 * (rank + 1)], [1000.0 * (rank + 1)],
                                         world, torch.device("cpu"))
        out[rank] = (mx, sm)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_the_summed_work():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        mx, sm = res[rank]
        assert mx == [11.0, 6.0]
        assert sm == [3000.0]


def test_one_rank_is_a_no_op():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks([1.5, 2.5], [7.0], 1, None) == ([1.5, 2.5], [7.0])
