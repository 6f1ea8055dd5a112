"""The multi-GPU form of the benchmark is weak scaling over independent
tensors: every rank takes its own tensors (no data-path collective) and the
job's time is the slowest rank's.  Checked here with world_size-2 gloo
process groups on the CPU (host logic only; no GPU)."""
import argparse
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ns = argparse.Namespace(pairs=16)
        specs = bench._batched_specs(rank, ns)
        seeds = [p[2][1].sum() for p in bench._pairs_small(rank, argparse.Namespace(pairs=2))]

        def reduce_max(v):
            t = torch.tensor([v], dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())

        local_ms = 100.0 * (rank + 1)  # rank 1 is the slow one
        value, ms = bench.job_value(local_ms, len(specs), 5, ws, reduce_max)
        gathered = [None] * ws
        dist.all_gather_object(gathered, (specs, seeds))
        out[rank] = (value, ms, gathered)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_take_disjoint_tensors_and_the_slowest_time():
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(ws, port, out), nprocs=ws, join=True, start_method="spawn")
    v0, ms0, g0 = out[0]
    v1, ms1, g1 = out[1]
    assert ms0 == ms1 == 200.0                       # max over ranks
    assert v0 == v1 == pytest.approx(2 * 16 * 5 / 0.2)  # all ranks' tensors / the slowest rank's time
    (s0, e0), (s1, e1) = g0
    assert len(s0) == len(s1) == 16
    assert not set(s0) & set(s1)                     # batched wave: disjoint tensors per rank
    assert set(e0).isdisjoint(set(e1))               # small pairs: different seeds per rank
