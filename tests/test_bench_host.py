"""Host logic of bench.py without a GPU: the whole-job aggregation of the multi-process launch
(every rank solves its own replica; the step time is the slowest rank's, all ranks' DoFs count),
run as two gloo ranks on CPU, and the lookup of the measured DRAM traffic record."""
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")  # rank 1 is the slow one
        out[rank] = (ms, bench.job_value(1000, world, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == 15.0
    assert abs(value - 2 * 1000 / 15e-3) < 1e-6


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_value(789507, 1, 10.0) == pytest.approx(78950700.0)


def test_traffic_record_lookup(tmp_path):
    import bench
    a = types.SimpleNamespace(dim=2, degree=2, split=1)
    h = bench.kernel_source_hash()
    (tmp_path / "x.md").write_text("text\ntraffic-record: kernel=k dim=2 degree=2 split=1 dofs=100 bytes=5000 "
                                   "source=%s\n" % h)
    assert bench.measured_traffic(a, 200, str(tmp_path)) == pytest.approx(10000.0)
    (tmp_path / "x.md").write_text("traffic-record: kernel=k dim=2 degree=2 split=1 dofs=100 bytes=5000 source=0\n")
    assert bench.measured_traffic(a, 200, str(tmp_path)) is None
    assert bench.measured_traffic(types.SimpleNamespace(dim=3, degree=2, split=1), 200, str(tmp_path)) is None


def test_algorithmic_bytes_per_dof():
    """Hand counts of the roofline's byte model: x and y once each, the per-point values of every
    Gauss point of a cell spread over the cell's DoFs, one flag byte per node."""
    import bench
    assert [bench.qp_values(2, s) for s in (0, 1)] == [7, 11]
    assert [bench.qp_values(3, s) for s in (0, 1)] == [10, 29]
    # 2D Q2 Miehe FP32: 8 + 11 * 9 * 4 / 12 + 1/3
    assert bench.apply_bytes_per_dof(2, 2, 1, 4) == pytest.approx(8 + 33 + 1 / 3)
    # 3D Q2 Miehe FP32: 8 + 29 * 27 * 4 / 32 + 1/4
    assert bench.apply_bytes_per_dof(3, 2, 1, 4) == pytest.approx(8 + 97.875 + 0.25)
    # FP64: twice the vector and per-point bytes
    assert bench.apply_bytes_per_dof(2, 2, 1, 8) == pytest.approx(16 + 66 + 1 / 3)


def test_method_minimum_bytes_per_dof():
    """The roofline's algorithmic bytes (SURVEY's method minimum): x and y once each, d + 2 state values
    per node over d + 1 DoFs per node, one flag byte per node."""
    import bench
    assert bench.method_bytes_per_dof(2, 4) == pytest.approx(8 + 16 / 3 + 1 / 3)   # 13.67
    assert bench.method_bytes_per_dof(2, 8) == pytest.approx(16 + 32 / 3 + 1 / 3)  # 27.0
    assert bench.method_bytes_per_dof(3, 4) == pytest.approx(8 + 20 / 4 + 1 / 4)   # 13.25
