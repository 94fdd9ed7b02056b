"""GPU parity of the exact discrete adjoint (rte_discrete_adjoint_gradient:
the reverse sweep of the discrete march with the transposed FC operators,
the transposed boundary map and readout, AB4 backwards) against the
oracle's reverse sweep on the same seeded inputs; the objective against the
oracle's; and the gradient against central differences of the library's own
objective, which the continuous adjoint only reaches to discretisation
level."""
import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2
from oracle.rte import Solver
from rte_inputs import workload_custom

pytestmark = pytest.mark.gpu

FP32, TF32X3, BF16X3 = 0, 1, 3
# FP32 passes and 3xTF32 carry FP32-level rounding through ~100 steps of the
# march and its transpose (observed below 1e-6); bf16x3 operands about 2^-16
# per product (observed 1.3e-5).
TOL = {FP32: 1e-5, TF32X3: 1e-5, BF16X3: 2e-4}


def _case(nx, ny, M, steps=90, groups=2):
    kw = dict(L=1.0, mua=0.35, mus=8.0, n_groups=groups, t_s=1.5, sigma_t=0.5)
    wl = workload_custom(nx, ny, M, steps, 0.04, heterogeneous=False, **kw)
    tgt = workload_custom(nx, ny, M, steps, 0.04, heterogeneous=True, **kw)
    St = Solver(tgt)
    meas = np.stack([St.forward(g, steps, tgt.detectors)["curves"] for g in tgt.groups]) * 0.8
    return wl, meas


def _gpu(wl, precision, ckpt, fc_parts=(1, 1), mua=None):
    from paper_2202_09421_gb300.solver import FCDOMSolver
    dev = torch.device("cuda:0")
    a = torch.tensor(wl.mua if mua is None else mua, dtype=torch.float32, device=dev)
    b = torch.tensor(wl.mus, dtype=torch.float32, device=dev)
    return FCDOMSolver(wl.grid, wl.optics, a, b, wl.c, wl.dt, ckpt_interval=ckpt, precision=precision,
                       fc_parts=fc_parts)


def _oracle(wl, meas, fc_parts=(1, 1)):
    S = Solver(wl, fc_parts=fc_parts)
    J, ga, gb = 0.0, 0.0, 0.0
    for k, g in enumerate(wl.groups):
        j, a_, b_ = S.discrete_adjoint_gradient(g, wl.n_steps, wl.detectors, meas[k])
        J, ga, gb = J + j, ga + a_, gb + b_
    return J, ga, gb


@pytest.mark.parametrize("nx,ny,M,precision,ckpt", [
    (40, 36, 16, FP32, 13), (40, 36, 16, TF32X3, 13), (40, 36, 16, BF16X3, 1000),
    (33, 35, 32, FP32, 1000), (33, 35, 32, TF32X3, 7)])
def test_discrete_adjoint_matches_oracle(nx, ny, M, precision, ckpt):
    wl, meas = _case(nx, ny, M)
    s = _gpu(wl, precision, ckpt)
    s.forward(wl.groups, wl.n_steps)
    m = torch.tensor(meas, dtype=torch.float32, device=s.device)
    J, ga, gb = s.discrete_adjoint_gradient(wl.detectors, m)
    s.close()
    Jo, gao, gbo = _oracle(wl, meas)
    ea, eb = rel_l2(ga.cpu(), gao), rel_l2(gb.cpu(), gbo)
    print(f"{nx}x{ny} M{M} prec {precision} ckpt {ckpt}: J {J:.6e} vs {Jo:.6e}; "
          f"dJ/da rel L2 {ea:.2e}; dJ/db rel L2 {eb:.2e}")
    assert abs(J - Jo) < 1e-5 * abs(Jo)
    assert ea < TOL[precision] and eb < TOL[precision]


def test_discrete_adjoint_subdomain_operator():
    """With the decomposed FC operator (Sec. 4.4) the sweep uses the
    transpose of the block operator."""
    wl, meas = _case(40, 36, 16, steps=60, groups=1)
    s = _gpu(wl, TF32X3, 20, fc_parts=(2, 2))
    s.forward(wl.groups, wl.n_steps)
    m = torch.tensor(meas, dtype=torch.float32, device=s.device)
    J, ga, gb = s.discrete_adjoint_gradient(wl.detectors, m)
    s.close()
    Jo, gao, gbo = _oracle(wl, meas, fc_parts=(2, 2))
    ea, eb = rel_l2(ga.cpu(), gao), rel_l2(gb.cpu(), gbo)
    print(f"parts (2, 2): dJ/da rel L2 {ea:.2e}; dJ/db rel L2 {eb:.2e}")
    assert abs(J - Jo) < 1e-5 * abs(Jo)
    assert ea < 1e-5 and eb < 1e-5


def test_discrete_adjoint_is_the_gradient_of_the_library_objective():
    """Central differences of the library's own J (FP64 objective of FP32
    curves) along a smooth direction: the discrete gradient matches them to
    the differences' rounding, the continuous adjoint only to its
    discretisation error."""
    wl, meas = _case(40, 36, 16, steps=90, groups=1)
    g = wl.grid
    X, Y = np.meshgrid(np.linspace(0, 1, g.nx), np.linspace(0, 1, g.ny))
    da = np.cos(2.1 * X + 0.3) * np.sin(1.7 * Y + 0.5)
    m = None

    def J_of(mua):
        nonlocal m
        s = _gpu(wl, TF32X3, 1000, mua=mua)
        m = torch.tensor(meas, dtype=torch.float32, device=s.device)
        s.forward(wl.groups, wl.n_steps)
        J = s.objective(wl.detectors, m)
        s.close()
        return J

    eps = 0.05
    fd = (J_of(wl.mua + eps * da) - J_of(wl.mua - eps * da)) / (2 * eps)
    s = _gpu(wl, TF32X3, 1000)
    s.forward(wl.groups, wl.n_steps)
    _, gd, _ = s.discrete_adjoint_gradient(wl.detectors, m)
    s.forward(wl.groups, wl.n_steps)
    _, gc, _ = s.adjoint_gradient(wl.detectors, m)
    s.close()
    dd = float((gd.double().cpu().numpy() * da).sum())
    dc = float((gc.double().cpu().numpy() * da).sum())
    print(f"central differences {fd:.6e}: discrete {dd:.6e} ({abs(dd - fd) / abs(fd):.1e}), "
          f"continuous {dc:.6e} ({abs(dc - fd) / abs(fd):.1e})")
    # FP32 rounding of J over the step (observed 4e-5 of the difference)
    assert abs(dd - fd) < 5e-4 * abs(fd)
    assert abs(dd - fd) < abs(dc - fd)


def test_autograd_function_exact_backward():
    """RTEObjective(exact=True): backward is the exact discrete gradient."""
    from paper_2202_09421_gb300.solver import RTEObjective
    wl, meas = _case(40, 36, 16, steps=60, groups=1)
    s = _gpu(wl, TF32X3, 20)
    a = torch.tensor(wl.mua, dtype=torch.float32, device=s.device, requires_grad=True)
    b = torch.tensor(wl.mus, dtype=torch.float32, device=s.device, requires_grad=True)
    m = torch.tensor(meas, dtype=torch.float32, device=s.device)
    J = RTEObjective.apply(a, b, m, s, wl.groups, wl.n_steps, wl.detectors, True)
    J.backward()
    J2, ga, gb = s.discrete_adjoint_gradient(wl.detectors, m)
    s.close()
    assert abs(J.item() - J2) < 1e-12 * abs(J2)
    assert torch.equal(a.grad, ga) and torch.equal(b.grad, gb)


def test_discrete_adjoint_per_cell_central_differences():
    """Per-cell check on 20 seeded cells: the exact discrete dJ/da at a cell
    against central differences of the library's J under a perturbation of
    that cell alone.  J is about 570 times the largest nodal gradient here,
    so the FP32 rounding of J (about 1e-8 of J between two solves) is
    divided by 2 eps g: cells are drawn among those whose gradient is at
    least 10% of the largest, and eps is half the background a (expected
    rounding share about 2e-4).  The same central differences in FP64 on the
    oracle are within 1e-5 of its exact gradient at this step (the
    truncation)."""
    wl, meas = _case(40, 36, 16, steps=90, groups=2)
    s = _gpu(wl, TF32X3, 30)
    m = torch.tensor(meas, dtype=torch.float32, device=s.device)
    s.forward(wl.groups, wl.n_steps)
    _, ga, _ = s.discrete_adjoint_gradient(wl.detectors, m)
    ga = ga.double().cpu().numpy()
    rng = np.random.default_rng(20)
    cand = np.flatnonzero(np.abs(ga).ravel() >= 0.1 * np.abs(ga).max())
    cells = rng.choice(cand, size=20, replace=False)
    eps = 0.5 * float(wl.mua.mean())
    worst = 0.0
    for flat in cells:
        j, i = np.unravel_index(flat, ga.shape)
        Js = []
        for sign in (1.0, -1.0):
            mua = wl.mua.copy()
            mua[j, i] += sign * eps
            s.set_medium(torch.tensor(mua, dtype=torch.float32, device=s.device),
                         torch.tensor(wl.mus, dtype=torch.float32, device=s.device))
            s.forward(wl.groups, wl.n_steps)
            Js.append(s.objective(wl.detectors, m))
        fd = (Js[0] - Js[1]) / (2 * eps)
        worst = max(worst, abs(fd - ga[j, i]) / abs(ga[j, i]))
    s.close()
    print(f"20 cells: worst relative difference {worst:.1e}")
    assert worst < 1e-3
