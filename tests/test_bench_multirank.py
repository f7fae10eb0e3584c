"""The bench's multi-rank path on CPU: two gloo ranks on 127.0.0.1.  Each
rank flashes its own shard (weak scaling, no data-path collective); the job
time is the maximum over ranks and the job value counts every rank's
mixtures."""
import importlib.util
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    b = _bench()
    mine = 10.0 + 5.0 * rank  # rank 1 is the slower one
    ms = b.job_ms(mine, dist, torch.device("cpu"))
    from paper_2205_03090_gb300 import workloads as wl
    cond = b.rank_conditions(wl.WORKLOADS["nc8_1e6"], 64, rank)
    out[rank] = (ms, float(cond.P.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ws = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    # every rank sees the slowest rank's time
    assert res[0][0] == res[1][0] == 15.0
    # the ranks flash different mixtures (their own shards)
    assert res[0][1] != res[1][1]
    b = _bench()
    assert b.job_value(1000, 2, 1.0, 15.0) == pytest.approx(2 * 1000 / 0.015)
    assert np.isnan(b.job_value(1000, 2, float("nan"), 15.0))


def test_single_rank_needs_no_collective():
    b = _bench()
    assert b.job_ms(12.5, None, None) == 12.5
