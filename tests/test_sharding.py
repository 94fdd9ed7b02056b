"""Source sharding of the gradient (eq. Gradsumq: the objective and its
gradient are sums over the generalized sources) on two and three gloo ranks
on CPU.  Each rank computes the oracle's continuous-adjoint gradient of its
contiguous share of the sources; one FP64 all-reduce adds the shares.  The
result equals the single-process gradient over all sources to FP64 rounding
(the sums differ only in their association)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    from rte_inputs import workload_custom
    wl = workload_custom(20, 18, 8, 40, 0.04, L=1.0, mua=0.35, mus=8.0, n_groups=5, heterogeneous=False,
                         t_s=1.0, sigma_t=0.4)
    tgt = workload_custom(20, 18, 8, 40, 0.04, L=1.0, mua=0.35, mus=8.0, n_groups=5, heterogeneous=True,
                          t_s=1.0, sigma_t=0.4)
    return wl, tgt


def _oracle_local(wl):
    from oracle.rte import Solver
    S = Solver(wl)

    def local_fn(groups, measured):
        J, ga, gb = 0.0, 0.0, 0.0
        for beams, meas in zip(groups, measured):
            j, a_, b_, _ = S.adjoint_gradient(beams, wl.n_steps, wl.detectors, np.asarray(meas))
            J, ga, gb = J + j, ga + a_, gb + b_
        return J, ga, gb
    return local_fn


def _measured(tgt):
    from oracle.rte import Solver
    St = Solver(tgt)
    return np.stack([St.forward(g, tgt.n_steps, tgt.detectors)["curves"] for g in tgt.groups])


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2202_09421_gb300.sharding import sharded_gradient
    wl, tgt = _case()
    J, ga, gb = sharded_gradient(wl.groups, _measured(tgt), _oracle_local(wl), (wl.grid.ny, wl.grid.nx))
    out[rank] = (J, ga.numpy(), gb.numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_gradient_equals_single_process(world):
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert set(out.keys()) == set(range(world))
    wl, tgt = _case()
    J, ga, gb = _oracle_local(wl)(wl.groups, _measured(tgt))
    assert abs(J) > 0 and np.abs(ga).max() > 0
    for r in range(world):
        Jr, gar, gbr = out[r]
        assert abs(Jr - J) <= 1e-13 * abs(J)
        assert np.abs(gar - ga).max() <= 1e-13 * np.abs(ga).max()
        assert np.abs(gbr - gb).max() <= 1e-13 * np.abs(gb).max()


def test_shard_ranges_partition_the_sources():
    from paper_2202_09421_gb300.sharding import shard_range
    for n in (0, 1, 4, 5, 16, 17):
        for world in (1, 2, 3, 8, 20):
            spans = [shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(4, 2, 2)
