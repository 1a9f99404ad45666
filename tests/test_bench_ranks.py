"""The benchmark's multi-process path on CPU: two gloo ranks, each with its own
replica timing; the whole-job value is the sum of the ranks' cell updates
over the slowest rank's time (no data-path collective)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    ranks = bench.Ranks()
    try:
        ranks.barrier()
        ms, value = bench.aggregate(10.0 * (rank + 1), 1000.0, 5, ranks)
        out[rank] = (ms, value)
    finally:
        ranks.close()


@pytest.mark.skipif(torch.cuda.is_available(), reason="CPU gloo check")
def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == pytest.approx(20.0)                     # slowest rank
        assert value == pytest.approx(world * 1000.0 * 5 / 0.020)


def _ref_worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.argv = ["bench.py", "--impl", "reference", "--workload", "landau16_f64", "--steps", "1",
                "--warmup", "0"]
    import bench
    ranks = bench.Ranks()
    try:
        res = bench.run_reference(bench.parse(), ranks)
        out[rank] = None if res is None else (res["impl"], res["value"], res["cpu_baseline"]["kind"])
    finally:
        ranks.close()


@pytest.mark.skipif(torch.cuda.is_available(), reason="CPU gloo check")
def test_reference_arm_runs_on_rank_0_only():
    """Under torchrun the reference arm (the oracle) runs on rank 0 alone; the
    other ranks return at once without work."""
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_ref_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[1] is None
    impl, value, kind = out[0]
    assert impl == "reference" and kind == "oracle" and value > 0
