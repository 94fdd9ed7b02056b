"""Source sharding across ranks (one GPU per rank) for the gradient of the
inverse problem.

Every generalized source q_i of eq. (RTEsources) -- a single beam in the
Transport Sweep, a group of staggered beams in the Multiple Staggered Source
scheme -- is an independent forward/adjoint pair; the objective and its
gradient are sums over the sources (eq. FObj and the gradient summed over i,
eq. Gradsumq).  So the only exchange a multi-GPU gradient needs is one sum:
each rank solves a contiguous share of the sources and the ranks add their
J, dJ/dmua and dJ/dmus in FP64 with a single all-reduce.  There is no
exchange inside a time step (no spatial decomposition, no halo).

The per-rank work is a callable ``local_fn(groups, measured) -> (J, dJ/dmua,
dJ/dmus)``; ``library_local_gradient`` binds it to the CUDA library."""
from __future__ import annotations

from typing import Callable, Sequence, Tuple

import numpy as np
import torch
import torch.distributed as dist

LocalFn = Callable[[Sequence, object], Tuple[float, object, object]]


def shard_range(n_groups: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous share [lo, hi) of n_groups sources for `rank` of `world`:
    the first n_groups % world ranks take one more (shares differ by at most
    one source, and some are empty when world > n_groups)."""
    if world < 1 or not 0 <= rank < world or n_groups < 0:
        raise ValueError("bad rank / world / group count")
    base, extra = divmod(n_groups, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def sharded_gradient(groups: Sequence, measured, local_fn: LocalFn, ncell_shape, process_group=None):
    """J, dJ/dmua, dJ/dmus over all `groups` with the work split across the
    ranks of `process_group` (the default group when None).

    measured is indexed [group][det][step] (a tensor or an array with the
    groups' data in order); rank r passes groups[lo:hi] and measured[lo:hi]
    to local_fn.  The three results are packed into one FP64 vector [J,
    dJ/dmua, dJ/dmus] and summed with a single all-reduce (on the device of
    the gradients for NCCL, on the host for gloo).  Ranks with no sources
    contribute zeros.  Every rank returns the full sums as (float, float64
    tensor, float64 tensor) of shape ncell_shape on the host."""
    world = dist.get_world_size(process_group)
    rank = dist.get_rank(process_group)
    lo, hi = shard_range(len(groups), rank, world)
    ncell = int(np.prod(ncell_shape))
    backend = dist.get_backend(process_group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    packed = torch.zeros(1 + 2 * ncell, dtype=torch.float64, device=dev)
    if hi > lo:
        J, ga, gb = local_fn(groups[lo:hi], measured[lo:hi])
        packed[0] = float(J)
        packed[1:1 + ncell] = torch.as_tensor(ga, dtype=torch.float64).reshape(-1).to(dev)
        packed[1 + ncell:] = torch.as_tensor(gb, dtype=torch.float64).reshape(-1).to(dev)
    dist.all_reduce(packed, op=dist.ReduceOp.SUM, group=process_group)
    packed = packed.cpu()
    return (float(packed[0]), packed[1:1 + ncell].reshape(ncell_shape),
            packed[1 + ncell:].reshape(ncell_shape))


def library_local_gradient(solver, n_steps: int, detectors, exact: bool = False) -> LocalFn:
    """local_fn for sharded_gradient on this rank's GPU: forward over the
    rank's groups, then the continuous adjoint of eq. (AdjointProblem) (or,
    with exact, the exact discrete adjoint), through the library's C ABI."""
    def local_fn(groups, measured):
        solver.forward(list(groups), n_steps)
        meas = torch.as_tensor(measured, dtype=torch.float32, device=solver.device).contiguous()
        fn = solver.discrete_adjoint_gradient if exact else solver.adjoint_gradient
        J, ga, gb = fn(detectors, meas)
        return J, ga.double(), gb.double()
    return local_fn
