"""Host logic of bench.py's multi-rank mode (one replica per GPU under torchrun), run as
two gloo ranks on the CPU: the environment is read as torchrun sets it and the step time
reported is the slowest rank's."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, lr = bench.dist_env()
        t = bench.max_over_ranks(1.0 + 0.5 * rank, w, "cpu")
        out[rank] = (w, r, lr, t)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (2, 0, 0, 1.5) and out[1] == (2, 1, 1, 1.5)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
