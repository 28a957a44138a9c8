"""The multi-rank harness of bench.py (N > 1: independent replicas, weak
scaling) on CPU: two gloo ranks rendezvous on 127.0.0.1, the step time is the
maximum over ranks and the whole-job value counts every rank's units."""
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


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (ws, rank, rank)
    dist.init_process_group("gloo")
    dist.barrier()
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
    m = bench.max_over_ranks(ms, w, "cpu")
    out[rank] = (m, bench.replica_value(1000, w, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_value():
    ws = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True)
    for rank in range(ws):
        m, v = out[rank]
        assert m == 15.0
        assert v == pytest.approx(2 * 1000 / 0.015)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.replica_value(72082790, 1, 0.5) == pytest.approx(72082790 / 0.0005)
