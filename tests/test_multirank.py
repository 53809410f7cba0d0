"""The multi-GPU path of the benchmark on CPU: two gloo ranks get disjoint wavelength
batches of independent problems, and the step time reported is the slowest rank's."""
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


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2408_14425_b300 import workloads
    lams = bench.rank_lambdas(rank, 4)
    chi, _ = workloads.grf_fields(32, 4, lambdas=lams)
    t = bench.max_over_ranks(10.0 + rank, dist)
    dist.barrier()
    out[rank] = (lams, float(chi.sum()), t)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_wavelengths_and_take_the_max_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    l0, s0, t0 = res[0]
    l1, s1, t1 = res[1]
    assert l0 == [0, 1, 2, 3] and l1 == [4, 5, 6, 7]
    assert not set(l0) & set(l1)
    assert s0 != s1                      # independent fields per rank
    assert t0 == t1 == 11.0              # the slowest rank's time on every rank


def test_single_rank_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.rank_lambdas(0, 64) == list(range(64))
