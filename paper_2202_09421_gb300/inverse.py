"""Inverse solver of Algorithm 2 (Sec. 5): the absorption field a(x) is the
minimiser of the objective of eq. (FObjpr) under the bounds
a_lower <= a <= a_upper (eq. minprob), found by the bound-constrained
limited-memory quasi-Newton method of Byrd, Lu, Nocedal and Zhu (L-BFGS-B,
the paper's lm-BFGS), each iteration driven by a forward and an adjoint
march per generalized source (the library's rte_forward and
rte_adjoint_gradient).  The optimiser is host logic (scipy's L-BFGS-B on
the nx*ny absorption values); every march runs in the CUDA library.

The loop is written against an `evaluate(a) -> (J, dJ/da)` callable, so
that the same iteration can be driven by the GPU solver (`gpu_evaluator`)
or, in the tests, by any other implementation of the same objective."""
from __future__ import annotations

import time

import numpy as np


def node_areas(grid) -> np.ndarray:
    """Trapezoid weight of every grid node ([ny][nx]): the quadrature of the
    integrals over the domain in eq. (errl2)."""
    dx = (grid.xmax - grid.xmin) / (grid.nx - 1)
    dy = (grid.ymax - grid.ymin) / (grid.ny - 1)
    wx = np.full(grid.nx, dx)
    wx[[0, -1]] *= 0.5
    wy = np.full(grid.ny, dy)
    wy[[0, -1]] *= 0.5
    return np.outer(wy, wx)


def relative_error(a, a_true, area) -> float:
    """E(i) of eq. (errl2): the L2 distance of the absorption iterate from
    the target, relative to the target's L2 norm."""
    a = np.asarray(a, dtype=np.float64)
    a_true = np.asarray(a_true, dtype=np.float64)
    num = float(np.sum(area * (a_true - a) ** 2))
    den = float(np.sum(area * a_true ** 2))
    return float(np.sqrt(num / den))


def gpu_evaluator(solver, groups, n_steps: int, detectors, measured, mus, exact: bool = False):
    """J(a) and dJ/da for the library: set the medium (a, mus), run the
    forward march of every group, then the checkpointed adjoint march
    (the solver needs a checkpoint interval): the paper's continuous
    adjoint, or with exact=True the exact gradient of the discrete objective.
    a is a host [ny][nx] array."""
    import torch

    dev = solver.device
    grad = solver.discrete_adjoint_gradient if exact else solver.adjoint_gradient

    def evaluate(a: np.ndarray):
        at = torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
        solver.set_medium(at, mus)
        solver.forward(groups, n_steps)
        J, ga, _ = grad(detectors, measured)
        return float(J), ga.double().cpu().numpy()

    return evaluate


def reconstruct(evaluate, a0, a_lower, a_upper, max_iter: int = 10, a_true=None, area=None,
                maxcor: int = 10):
    """Runs L-BFGS-B from a0 (host [ny][nx]) within [a_lower, a_upper]
    (scalars or arrays of the same shape) for at most max_iter iterations.
    The objective is normalised by its value at a0 (the relative scale of J
    is what the stopping rules see).  Returns a dict with the final field,
    the number of objective evaluations and, per iteration, J, E(i) (when
    a_true and area are given) and the elapsed wall time."""
    from scipy.optimize import minimize

    a0 = np.asarray(a0, dtype=np.float64)
    shape = a0.shape
    lo = np.broadcast_to(np.asarray(a_lower, dtype=np.float64), shape).ravel()
    hi = np.broadcast_to(np.asarray(a_upper, dtype=np.float64), shape).ravel()
    scale = {}
    count = {"nfev": 0}
    last = {}

    def fg(x):
        if "x" in last and np.array_equal(last["x"], x):      # the same point again
            J, g = last["J"], last["g"]
        else:
            J, g = evaluate(x.reshape(shape))
            g = np.asarray(g, dtype=np.float64).ravel()
            count["nfev"] += 1
            last["x"], last["J"], last["g"] = x.copy(), J, g
        if "J0" not in scale:
            scale["J0"] = J if J > 0 else 1.0
        return J / scale["J0"], g / scale["J0"]

    history = []
    t0 = time.perf_counter()
    J_start, _ = fg(a0.ravel())
    history.append({"iteration": 0, "J": J_start * scale["J0"],
                    "E": relative_error(a0, a_true, area) if a_true is not None else None,
                    "seconds": time.perf_counter() - t0})

    def callback(xk):
        # the accepted iterate is the line search's last evaluation
        J = last["J"] if np.array_equal(last.get("x"), xk) else None
        rec = {"iteration": len(history), "J": J, "seconds": time.perf_counter() - t0}
        if a_true is not None:
            rec["E"] = relative_error(xk.reshape(shape), a_true, area)
        history.append(rec)

    res = minimize(fg, a0.ravel(), jac=True, method="L-BFGS-B", bounds=list(zip(lo, hi)), callback=callback,
                   options={"maxiter": max_iter, "maxcor": maxcor, "ftol": 1e-14, "gtol": 1e-14})
    return {"a": res.x.reshape(shape), "history": history, "nfev": count["nfev"], "message": str(res.message),
            "J_final": float(res.fun) * scale["J0"]}
