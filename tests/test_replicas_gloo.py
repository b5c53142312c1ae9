"""Host logic of the multi-rank bench (one independent tensor per rank, no collective on
the data path, max-over-ranks timing), run as two gloo ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        assert bench._dist() == (world, rank)
        slowest = bench._max_over_ranks(10.0 + 5.0 * rank, torch.device("cpu"))
        w = bench._workload(rank, "uniform5-n30")
        q.put((rank, slowest, w.nnz, int(np.asarray(w.idx, dtype=np.int64).sum()), float(w.vals.sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_distinct_tensors():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    assert [o[1] for o in out] == [15.0, 15.0]          # max over ranks, seen by every rank
    assert out[0][2] == out[1][2]                         # same size of problem per rank (weak scaling)
    assert (out[0][3], out[0][4]) != (out[1][3], out[1][4])   # an independent tensor per rank


def test_single_process_max_is_the_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.5, torch.device("cpu")) == 3.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.argparse.Namespace(gpus=2, steps=1, warmup=0)
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
