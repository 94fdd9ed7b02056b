"""GPU parity of the adjoint gradient (checkpointed recompute, adjoint march,
FP64 gradient accumulation) against the oracle's adjoint on the same inputs,
and of the objective J; autograd wrapper consistency."""
import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2
from oracle.rte import Solver
from rte_inputs import workload_custom

pytestmark = pytest.mark.gpu


def _setup(n=32, M=16, steps=150, groups=2, ckpt=40):
    wl = workload_custom(n, n, M, steps, 0.04, L=1.0, mua=0.35, mus=8.0, n_groups=groups,
                         heterogeneous=False, t_s=1.5, sigma_t=0.5)
    tgt = workload_custom(n, n, M, steps, 0.04, L=1.0, mua=0.35, mus=8.0, n_groups=groups,
                          heterogeneous=True, t_s=1.5, sigma_t=0.5)
    St = Solver(tgt)
    meas = np.stack([St.forward(g, steps, tgt.detectors)["curves"] for g in tgt.groups])
    return wl, meas


@pytest.mark.parametrize("ckpt", [40, 7, 1000])
def test_adjoint_gradient_matches_oracle(ckpt):
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl, meas = _setup(ckpt=ckpt)
    dev = torch.device("cuda:0")
    s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                    torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt,
                    ckpt_interval=ckpt)
    s.forward(wl.groups, wl.n_steps)
    m = torch.tensor(meas, dtype=torch.float32, device=dev)
    J, ga, gb = s.adjoint_gradient(wl.detectors, m)
    J_only = s.objective(wl.detectors, m)
    S = Solver(wl)
    Jo, gao, gbo = 0.0, 0.0, 0.0
    for k, g in enumerate(wl.groups):
        j, a_, b_, _ = S.adjoint_gradient(g, wl.n_steps, wl.detectors, meas[k])
        Jo, gao, gbo = Jo + j, gao + a_, gbo + b_
    print(f"ckpt {ckpt}: J {J:.6e} vs {Jo:.6e}; grad_a rel L2 {rel_l2(ga.cpu(), gao):.2e}; "
          f"grad_b rel L2 {rel_l2(gb.cpu(), gbo):.2e}")
    assert abs(J - Jo) < 1e-5 * abs(Jo) and abs(J_only - J) < 1e-12 * abs(J)
    assert rel_l2(ga.cpu(), gao) < 1e-4 and rel_l2(gb.cpu(), gbo) < 1e-4
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_gradient_m64_matches_oracle(precision):
    """M = 64: the gradient terms take the one-warp-per-cell form (the
    one-thread-per-cell form covers M = 16 and 32), in the plain FP32 and the
    3xTF32 precisions."""
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl, meas = _setup(n=24, M=64, steps=80, ckpt=30)
    dev = torch.device("cuda:0")
    s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                    torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt,
                    ckpt_interval=30, precision=precision)
    s.forward(wl.groups, wl.n_steps)
    J, ga, gb = s.adjoint_gradient(wl.detectors, torch.tensor(meas, dtype=torch.float32, device=dev))
    s.close()
    S = Solver(wl)
    Jo, gao, gbo = 0.0, 0.0, 0.0
    for k, g in enumerate(wl.groups):
        j, a_, b_, _ = S.adjoint_gradient(g, wl.n_steps, wl.detectors, meas[k])
        Jo, gao, gbo = Jo + j, gao + a_, gbo + b_
    print(f"M64 prec {precision}: J {J:.6e} vs {Jo:.6e}; grad_a rel L2 {rel_l2(ga.cpu(), gao):.2e}; "
          f"grad_b rel L2 {rel_l2(gb.cpu(), gbo):.2e}")
    assert abs(J - Jo) < 1e-5 * abs(Jo)
    assert rel_l2(ga.cpu(), gao) < 1e-4 and rel_l2(gb.cpu(), gbo) < 1e-4


def test_autograd_function_backward_is_the_adjoint():
    from paper_2202_09421_gb300.solver import FCDOMSolver, RTEObjective
    wl, meas = _setup(groups=1)
    dev = torch.device("cuda:0")
    a = torch.tensor(wl.mua, dtype=torch.float32, device=dev, requires_grad=True)
    b = torch.tensor(wl.mus, dtype=torch.float32, device=dev, requires_grad=True)
    m = torch.tensor(meas, dtype=torch.float32, device=dev)
    s = FCDOMSolver(wl.grid, wl.optics, a.detach(), b.detach(), wl.c, wl.dt, ckpt_interval=50)
    J = RTEObjective.apply(a, b, m, s, wl.groups, wl.n_steps, wl.detectors)
    J.backward()
    J2, ga, gb = s.adjoint_gradient(wl.detectors, m)
    assert abs(J.item() - J2) < 1e-12 * abs(J2)
    assert torch.allclose(a.grad, ga) and torch.allclose(b.grad, gb)
    s.close()


def test_sharded_gradient_through_the_library_on_one_rank():
    """sharded_gradient with the library's per-rank solve (a one-rank gloo
    group): the shares and the FP64 all-reduce give the same J and gradient
    as one rte_adjoint_gradient over all groups."""
    import socket

    import torch.distributed as dist

    from paper_2202_09421_gb300.sharding import library_local_gradient, sharded_gradient
    from paper_2202_09421_gb300.solver import FCDOMSolver
    from rte_inputs import workload_custom
    wl = workload_custom(40, 36, 16, 60, 0.04, L=1.0, mua=0.35, mus=8.0, n_groups=3, heterogeneous=False,
                         t_s=1.0, sigma_t=0.4)
    dev = torch.device("cuda:0")
    meas = torch.zeros((3, len(wl.detectors), wl.n_steps), dtype=torch.float32, device=dev)
    s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                    torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt, ckpt_interval=20)
    s.forward(wl.groups, wl.n_steps)
    J, ga, gb = s.adjoint_gradient(wl.detectors, meas)
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        Js, gas, gbs = sharded_gradient(wl.groups, meas, library_local_gradient(s, wl.n_steps, wl.detectors),
                                        (wl.grid.ny, wl.grid.nx))
    finally:
        dist.destroy_process_group()
    s.close()
    assert abs(Js - J) <= 1e-12 * abs(J)
    assert np.array_equal(gas.numpy(), ga.double().cpu().numpy())
    assert np.array_equal(gbs.numpy(), gb.double().cpu().numpy())
