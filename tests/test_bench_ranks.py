"""bench.py's multi-rank aggregation on two gloo ranks (CPU): the timed region is the
slowest rank's, the work (LPs solved, ADMM updates) is summed over the ranks."""
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    per_rank = {0: (2.0, 1, 1000), 1: (3.5, 0, 1200)}
    total_s, solved, admm = bench.aggregate_ranks(*per_rank[rank], dist, "cpu")
    out[rank] = (total_s, solved, admm, admm / total_s)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        total_s, solved, admm, value = out[r]
        assert total_s == 3.5
        assert solved == 1
        assert admm == 2200
        assert value == pytest.approx(2200 / 3.5)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(1.5, 2, 300) == (1.5, 2.0, 300.0)
