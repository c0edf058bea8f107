"""The multi-process path of bench.py on CPU: two ranks over the gloo backend (127.0.0.1).

With N replicas every rank solves its own instances and the job's time per step is that of
the slowest rank; bench.max_over_ranks takes that maximum with one all-reduce.  The test runs
it on two CPU processes with different values and checks that both ranks get the maximum, and
that one process (no process group) returns its own value.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, values, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(values[rank], dist, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()
    out[rank] = got


def test_max_over_ranks_gloo_two_ranks():
    import torch.multiprocessing as mp
    values = [0.0187, 0.0213]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, _free_port(), values, out), nprocs=2, join=True)
        assert out[0] == pytest.approx(max(values)) and out[1] == pytest.approx(max(values))


def test_max_over_ranks_one_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.5, None, "cpu") == 0.5
