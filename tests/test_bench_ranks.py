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


def test_traffic_model_is_keyed_on_the_measured_sources():
    """roofline.traffic comes from the ncu model only while the kernel sources hash to the
    measured ones, and scales with the update count: fixed + per-update bytes."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.TRAFFIC["sources_sha256"] == bench.kernel_sources_hash()
    t20, t60 = bench.traffic_per_launch(20), bench.traffic_per_launch(60)
    assert t60 - t20 == 40 * bench.TRAFFIC["dram_bytes_per_update"]
    saved = dict(bench.TRAFFIC)
    try:
        bench.TRAFFIC["sources_sha256"] = "0" * 64
        assert bench.traffic_per_launch(20) is None
    finally:
        bench.TRAFFIC.update(saved)


def test_algorithmic_bytes_follow_the_minimum_passes():
    """Per update: one pass over A and one over A^T plus 20 n-vectors; per PCG iteration two
    passes plus 6 m-vectors; a pass over a CSR matrix reads nnz (value + index) + row
    pointers."""
    sys.path.insert(0, ROOT)
    import bench
    m, n, nnz = 1000, 4000, 25000
    one = bench.algorithmic_bytes(m, n, nnz, admm_iters=1, cg_iters=0, vec_bytes=4)
    two = bench.algorithmic_bytes(m, n, nnz, admm_iters=2, cg_iters=0, vec_bytes=4)
    assert two == 2 * one
    cg = bench.algorithmic_bytes(m, n, nnz, admm_iters=0, cg_iters=1, vec_bytes=4)
    pass_a = nnz * (4 + 4) + 8 * (m + 1)
    pass_at = nnz * (4 + 4) + 8 * (n + 1)
    assert cg == pass_a + pass_at + 6 * m * 4
    assert one == pass_a + pass_at + 20 * n * 4


def test_both_arms_print_one_workload_config(monkeypatch):
    """The reference arm and the GPU arm build `config` from the same helper, so a ratio of
    the two lines compares the same LP and the same solver parameters."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--max-admm", "300", "--gamma", "0.2"])
    args = bench.parse()
    cfg = bench.workload_config(args, 1000, 4000, 25000, 1)
    assert cfg["workload"] == bench.WORKLOAD
    assert (cfg["m"], cfg["n"], cfg["nnz"]) == (1000, 4000, 25000)
    assert cfg["admm_updates_per_step"] == 300 and cfg["gamma"] == 0.2
    assert cfg["parallelism"] == "replicas1" and "flushed" in cfg["l2"]
    assert bench.workload_config(args, 1000, 4000, 25000, 1) == cfg
