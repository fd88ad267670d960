"""The multi-GPU path of the benchmark is replicas only: every rank runs its
own design and the ranks only agree on timing (a barrier and the MAX of the
per-rank times).  Checked here with two CPU ranks over gloo."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W
    wl = W.ORTHO_128
    seed = bench.replica_seed(wl, rank)
    rho = W.initial_density(16, wl.volfrac, seed)
    ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, world, "cpu")
    rate = bench.aggregate_rate(40, world, ms_max * 1e-3)
    dist.barrier()
    out.put((rank, seed, float(rho.sum()), ms_max, rate))
    dist.destroy_process_group()


def test_two_replicas_agree_on_timing_and_differ_in_design():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, max0, rate0), (r1, s1, m1, max1, rate1) = res
    assert s0 != s1 and m0 != m1                 # independent designs
    assert max0 == max1 == 15.0                  # the slowest rank's time on every rank
    assert rate0 == rate1 == pytest.approx(2 * 40 / 0.015)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.aggregate_rate(10, 1, 2.0) == 5.0
