"""The multi-GPU path of bench.py is replicas only: each rank runs the whole
workload, the timings are maximised over the ranks, and the JSON value is
the units of all ranks over the slowest rank's time.  Checked here with two
gloo ranks on the CPU (no GPU)."""
import os
import socket

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
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.replica_times([1.0 + rank, 10.0 - rank, 0.5 * (rank + 1)], dist)
    out[rank] = t + [bench.replica_value(100.0, world, t[0])]
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == [2.0, 10.0, 1.0, 100.0]


def test_one_rank_is_unchanged():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_times([0.25, 3], None) == [0.25, 3.0]
    assert bench.replica_value(48.0, 1, 2.0) == 24.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the oracle arm prints from rank 0 alone; other ranks
    return at once without work."""
    import sys
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    a = argparse.Namespace(workload="al108_48", gpus=2, steps=1, warmup=3, cpu_sample=0)
    assert bench.run_reference(a) is None
    assert capsys.readouterr().out == ""
