"""The N > 1 path of bench.py is replicas only: each rank solves its own
field and the job's time is the slowest rank's, its work the sum.  Checked
with two gloo ranks on the CPU (no GPU, no data-path collective)."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from bench import aggregate_replicas
        t, u = aggregate_replicas(10.0 + 5.0 * rank, 1000 * (rank + 1), world, None)
        out[rank] = (t, u)
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (15.0, 3000.0)


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    from bench import aggregate_replicas
    assert aggregate_replicas(7.5, 42, 1) == (7.5, 42.0)
