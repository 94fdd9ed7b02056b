"""Python-side convenience around the C ABI: a solver object holding one
context, and a torch.autograd.Function whose backward is the library's
checkpointed adjoint march (Sec. 3.4-3.6).  Marshalling only."""
from __future__ import annotations

import torch

from . import binding as B


class FCDOMSolver:
    """One medium on one grid.  grid/optics are duck-typed (nx, ny, xmin, xmax,
    ymin, ymax, M / g, n_in, n_out, hg_exponent); c is the speed of light in
    the medium (cm/ps)."""

    def __init__(self, grid, optics, mua: torch.Tensor, mus: torch.Tensor, c: float, dt: float,
                 ckpt_interval: int = 0, filter_alpha: float = 2.0, filter_beta: float = 55.0,
                 stream=None, precision: int = 0, flags: int = 0, fc_parts=(1, 1)):
        self.grid = grid
        self.device = mua.device

        class _Opt:
            pass
        o = _Opt()
        o.g, o.n_in, o.n_out = optics.g, optics.n_in, optics.n_out
        o.hg_exponent, o.c = optics.hg_exponent, c
        params = B.RteParams(dt, filter_alpha, filter_beta, int(ckpt_interval), int(precision), int(flags),
                             int(fc_parts[0]), int(fc_parts[1]))
        self.ctx = B.rte_init_medium(grid, mua.contiguous(), mus.contiguous(), o, params, stream)
        self.n_groups = 0
        self.n_steps = 0

    def set_medium(self, mua, mus):
        B.rte_set_medium(self.ctx, mua.contiguous(), mus.contiguous())

    def forward(self, groups, n_steps: int, snap_steps=()):
        g = self.grid
        fl = None
        if snap_steps:
            fl = torch.empty((len(groups), len(snap_steps), g.ny, g.nx), device=self.device,
                             dtype=torch.float32)
        B.rte_forward(self.ctx, groups, n_steps, list(snap_steps), fl)
        self.n_groups, self.n_steps = len(groups), n_steps
        return fl

    def readout(self, detectors) -> torch.Tensor:
        out = torch.empty((self.n_groups, len(detectors), self.n_steps), device=self.device,
                          dtype=torch.float32)
        B.rte_detector_readout(self.ctx, detectors, out)
        return out

    def objective(self, detectors, measured) -> float:
        return B.rte_objective(self.ctx, detectors, measured.contiguous())

    def adjoint_gradient(self, detectors, measured):
        g = self.grid
        ga = torch.empty((g.ny, g.nx), device=self.device, dtype=torch.float32)
        gb = torch.empty_like(ga)
        J = B.rte_adjoint_gradient(self.ctx, detectors, measured.contiguous(), ga, gb)
        return J, ga, gb

    def discrete_adjoint_gradient(self, detectors, measured):
        """J and its exact gradient with respect to the nodal a and b of the
        discrete march (the reverse sweep with the transposed operators)."""
        g = self.grid
        ga = torch.empty((g.ny, g.nx), device=self.device, dtype=torch.float32)
        gb = torch.empty_like(ga)
        J = B.rte_discrete_adjoint_gradient(self.ctx, detectors, measured.contiguous(), ga, gb)
        return J, ga, gb

    def photon_balance(self) -> torch.Tensor:
        """[group][step][3] float64: photons int Phi / c, absorption rate
        int a Phi, net outward boundary flux of every step of the last
        forward (the solver needs flags with RTE_FLAG_PHOTON_BALANCE)."""
        out = torch.empty((self.n_groups, self.n_steps, 3), device=self.device, dtype=torch.float64)
        B.rte_photon_balance(self.ctx, out)
        return out

    def state(self, group: int) -> torch.Tensor:
        g = self.grid
        out = torch.empty((g.ny, g.nx, g.M), device=self.device, dtype=torch.float32)
        B.rte_get_state(self.ctx, group, out)
        return out

    def kernel_launches(self) -> int:
        return B.rte_kernel_launches(self.ctx)

    def graph_captures(self) -> int:
        return B.rte_graph_captures(self.ctx)

    def autotune(self, groups, n_trial_steps: int = 40):
        """Times the kernel configurations of this precision on these groups
        and keeps the fastest; returns (choice, {choice: ms})."""
        return B.rte_autotune(self.ctx, groups, n_trial_steps)

    def close(self):
        if self.ctx is not None:
            B.rte_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def forward_batch(solvers, groups_per_solver, n_steps: int):
    """Advances several solvers (media of their own grid sizes, same M,
    precision, flags and stream) through one forward march in lockstep
    (rte_forward_batch); afterwards readout/objective/adjoint_gradient apply
    per solver."""
    B.rte_forward_batch([s.ctx for s in solvers], groups_per_solver, n_steps)
    for s, groups in zip(solvers, groups_per_solver):
        s.n_groups, s.n_steps = len(groups), n_steps


def adjoint_gradient_batch(solvers, detectors_per_solver, measured_per_solver):
    """The continuous adjoint of every solver after a march of the same steps
    (rte_adjoint_gradient_batch): a list of (J, dJ/dmua, dJ/dmus) per solver."""
    gas = [torch.empty((s.grid.ny, s.grid.nx), device=s.device, dtype=torch.float32) for s in solvers]
    gbs = [torch.empty_like(g) for g in gas]
    Js = B.rte_adjoint_gradient_batch([s.ctx for s in solvers], detectors_per_solver,
                                      [m.contiguous() for m in measured_per_solver], gas, gbs)
    return list(zip(Js, gas, gbs))


class RTEObjective(torch.autograd.Function):
    """J(mua, mus) = sum over groups of eq. (FObj) for the given beams and
    detectors.  forward: rte_forward + rte_objective; backward: the adjoint
    march of eq. (AdjointProblem) with checkpoint recompute, giving dJ/dmua
    and dJ/dmus per grid node (eq. FDwin22), or, with exact=True, the
    exact gradient of the discrete objective (the reverse sweep of the
    march, rte_discrete_adjoint_gradient)."""

    @staticmethod
    def forward(ctx, mua, mus, measured, solver: FCDOMSolver, groups, n_steps, detectors, exact=False):
        solver.set_medium(mua.detach(), mus.detach())
        solver.forward(groups, n_steps)
        J = solver.objective(detectors, measured)
        ctx.solver, ctx.detectors, ctx.exact = solver, detectors, exact
        ctx.save_for_backward(measured)
        return torch.tensor(J, dtype=torch.float64, device=mua.device)

    @staticmethod
    def backward(ctx, gJ):
        (measured,) = ctx.saved_tensors
        grad = ctx.solver.discrete_adjoint_gradient if ctx.exact else ctx.solver.adjoint_gradient
        _, ga, gb = grad(ctx.detectors, measured)
        scale = gJ.to(torch.float32)
        return scale * ga, scale * gb, None, None, None, None, None, None
