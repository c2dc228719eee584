"""The N > 1 path of bench.py on the CPU: two gloo ranks.

Ranks run independent replica batches (weak scaling, no data-path
collective): each rank draws its own replicas, the timing is the maximum
over ranks and the particle count the sum.  The reference arm runs on rank 0
only.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    system, run = bench.make_workload("batched", rank, 3)
    ms = 10.0 + 5.0 * rank
    t_max, n_total = bench.reduce_over_ranks(dist, ms, system.n, "cpu")
    # every rank's replicas, gathered for the check (test only)
    pos = torch.tensor(system.pos[:8].ravel())
    allpos = [torch.zeros_like(pos) for _ in range(world)]
    dist.all_gather(allpos, pos)
    ns = torch.tensor([float(system.n)])
    alln = [torch.zeros_like(ns) for _ in range(world)]
    dist.all_gather(alln, ns)
    out.put((rank, t_max, n_total, [p.numpy() for p in allpos], [float(x) for x in alln],
             run["ensemble"]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, t_max, n_total, allpos, alln, ens in res:
        assert t_max == 15.0                        # max over ranks
        assert n_total == int(sum(alln))            # whole-job particle count
        assert ens == "nvt"
        # the two ranks drew different replicas (seeds offset by rank)
        assert not np.allclose(allpos[0], allpos[1])


def test_reference_arm_other_ranks_do_nothing():
    import argparse
    import bench
    a = argparse.Namespace(impl="reference", workload="batched", replicas=512, steps=1,
                           warmup=0, gpus=2)
    assert bench.reference_arm(a, world=2, rank=1) is None


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(None, 12.5, 1000, "cpu") == (12.5, 1000)
