"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank
runs its own replica, the job's time is the maximum over ranks and the
whole-job throughput counts every replica's iterations."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench._dist() == (ws, rank, rank)
    ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    job_ms = bench.max_over_ranks(ms, ws, device="cpu")
    out[rank] = (job_ms, bench.job_value(ws, 5, job_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_is_max_over_ranks():
    ws = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0] == res[1]
    job_ms, value = res[0]
    assert job_ms == pytest.approx(20.0)
    assert value == pytest.approx(2 * 5 / 0.020)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_value(1, 10, 1000.0) == pytest.approx(10.0)
