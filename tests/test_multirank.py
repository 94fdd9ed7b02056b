"""The N > 1 path of bench.py on CPU: two gloo ranks.  Each rank solves the
whole workload on its own device (weak scaling, no collective on the data
path); the only collective is the max over ranks of the timed region, and
the reported rate counts every rank's updates.  Here each rank times a small
FP64 oracle solve in place of the GPU solve."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import time

    import numpy as np
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from oracle.rte import Solver
    from rte_inputs import workload_custom

    wl = workload_custom(24, 24, 8, 10 + 5 * rank, 0.04)      # ranks do different amounts of work
    t0 = time.perf_counter()
    curves = Solver(wl).forward(wl.groups[0], wl.n_steps, wl.detectors)["curves"]
    local_ms = (time.perf_counter() - t0) * 1e3
    updates = wl.grid.nx * wl.grid.ny * wl.grid.M * 10       # units each rank is credited with

    def max_fn(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    value, ms = bench.aggregate(updates, local_ms, world, max_fn)
    all_ms = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(all_ms, torch.tensor([local_ms], dtype=torch.float64))
    out[rank] = (value, ms, max(float(t) for t in all_ms), bool(np.isfinite(curves).all()))
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregate():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert set(out.keys()) == {0, 1}
    for r in range(world):
        value, ms, max_ms, finite = out[r]
        assert finite
        assert ms == pytest.approx(max_ms)                   # every rank sees the max time
        assert value == pytest.approx(24 * 24 * 8 * 10 * world / (max_ms / 1e3))
    assert out[0][0] == pytest.approx(out[1][0])
