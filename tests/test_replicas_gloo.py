"""The multi-GPU form is replicas only (no data-path collective): bench.py times
each rank and reports the slowest rank's step and the whole-job pairs/s.  The
host logic runs here on two CPU ranks over gloo."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t = bench.max_over_ranks(times[rank], torch.device("cpu"), ws)
    out[rank] = (t, bench.job_value(1.0e9, ws, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ws = 2
    times = [0.25, 0.40]
    with mp.get_context("spawn").Manager() as m:  # no fork: the parent may hold CUDA state
        out = m.dict()
        mp.spawn(_rank, args=(ws, _free_port(), times, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        t, v = res[r]
        assert t == 0.40
        assert v == pytest.approx(2 * 1.0e9 / 0.40)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(0.3, torch.device("cpu"), 1) == 0.3
    assert bench.job_value(5.0, 1, 0.5) == 10.0
