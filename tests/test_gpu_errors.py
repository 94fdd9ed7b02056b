"""Failure detection through the C ABI's status codes, with every fault made
on the host (no GPU fault, trap or hang): bad media, a time step outside the
AB4 stability estimate, calls out of order, invalid beams.  After each
rejected call the context still solves correctly."""
import dataclasses

import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2
from oracle.rte import Solver
from rte_inputs import workload_custom

pytestmark = pytest.mark.gpu

INVALID_ARG, UNSTABLE_DT, STATE = 1, 2, 6


def _wl():
    return workload_custom(32, 32, 16, 40, 0.04, L=1.0, mus=20.0, n_groups=1, t_s=1.0, sigma_t=0.4)


def _t(x):
    return torch.tensor(x, dtype=torch.float32, device="cuda:0")


def _status(fn, *args):
    from paper_2202_09421_gb300.binding import RTEError
    with pytest.raises(RTEError) as e:
        fn(*args)
    return e.value.status


def test_bad_media_and_unstable_dt_are_rejected():
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl = _wl()
    a, b = np.asarray(wl.mua, dtype=np.float64), np.asarray(wl.mus, dtype=np.float64)
    nan_a = a.copy()
    nan_a[5, 7] = np.nan
    neg_b = b.copy()
    neg_b[3, 3] = -1.0
    mk = lambda aa, bb, dt: FCDOMSolver(wl.grid, wl.optics, _t(aa), _t(bb), wl.c, dt)
    assert _status(mk, nan_a, b, wl.dt) == INVALID_ARG
    assert _status(mk, a, neg_b, wl.dt) == INVALID_ARG
    assert _status(mk, a, b, 50.0) == UNSTABLE_DT               # far outside the AB4 region
    # a medium change that would make the step unstable is refused and the
    # context keeps its medium
    s = mk(a, b, wl.dt)
    assert _status(s.set_medium, _t(a), _t(np.full_like(b, 1e5))) == UNSTABLE_DT
    s.forward(wl.groups, wl.n_steps)
    curves = s.readout(wl.detectors).cpu().numpy()
    s.close()
    ref = Solver(wl).forward(wl.groups[0], wl.n_steps, wl.detectors)["curves"]
    assert rel_l2(curves[0], ref) < 1e-5


def test_calls_out_of_order_and_invalid_beams():
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl = _wl()
    s = FCDOMSolver(wl.grid, wl.optics, _t(wl.mua), _t(wl.mus), wl.c, wl.dt, ckpt_interval=0)
    meas = torch.zeros((1, len(wl.detectors), wl.n_steps), dtype=torch.float32, device="cuda:0")
    from paper_2202_09421_gb300 import binding as B
    out = torch.empty((1, len(wl.detectors), wl.n_steps), dtype=torch.float32, device="cuda:0")
    assert _status(B.rte_detector_readout, s.ctx, wl.detectors, out) == STATE       # no forward yet
    bad = [[dataclasses.replace(wl.groups[0][0], sigma_x=0.0)]]
    assert _status(s.forward, bad, wl.n_steps) == INVALID_ARG
    s.forward(wl.groups, wl.n_steps)
    assert _status(s.adjoint_gradient, wl.detectors, meas) == STATE          # no checkpoints kept
    assert _status(s.discrete_adjoint_gradient, wl.detectors, meas) == STATE
    curves = s.readout(wl.detectors).cpu().numpy()
    s.close()
    ref = Solver(wl).forward(wl.groups[0], wl.n_steps, wl.detectors)["curves"]
    assert rel_l2(curves[0], ref) < 1e-5


# ---------------------------------------------------------------- timeout path
TIMEOUT, UNSUPPORTED = 5, 7
TF32X3 = 1


def _tc_solver(wl, **kw):
    from paper_2202_09421_gb300.solver import FCDOMSolver
    return FCDOMSolver(wl.grid, wl.optics, _t(wl.mua), _t(wl.mus), wl.c, wl.dt, precision=TF32X3, **kw)


def _oracle_curves(wl):
    return Solver(wl).forward(wl.groups[0], wl.n_steps, wl.detectors)["curves"]


def test_timeout_word_stops_the_march_and_is_cleared():
    """A set timeout word (as left by a bounded wait that ran out) makes every
    tensor-core pass of the march return at once: the call reports TIMEOUT
    and the state stays at its zero start.  The word is cleared with the
    report, and the next march on the same context matches the oracle."""
    from paper_2202_09421_gb300 import binding as B
    wl = _wl()
    s = _tc_solver(wl)
    B.rte_inject_fault(s.ctx, B.RTE_FAULT_TIMEOUT_WORD)
    assert _status(s.forward, wl.groups, wl.n_steps) == TIMEOUT
    state = torch.empty((wl.grid.ny, wl.grid.nx, wl.grid.M), dtype=torch.float32, device="cuda:0")
    B.rte_get_state(s.ctx, 0, state)
    assert float(state.abs().max()) == 0.0                        # no pass did any work
    s.forward(wl.groups, wl.n_steps)
    curves = s.readout(wl.detectors).cpu().numpy()
    s.close()
    assert rel_l2(curves[0], _oracle_curves(wl)) < 1e-5


def test_expiring_device_wait_reports_timeout():
    """One CTA of the first pass waits on a barrier that nothing arrives on
    (before it issues any copy or MMA): the bounded wait runs out (about
    2 s), the march reports TIMEOUT, and the context then solves correctly."""
    from paper_2202_09421_gb300 import binding as B
    wl = _wl()
    s = _tc_solver(wl)
    B.rte_set_pass_variant(s.ctx, 1)
    B.rte_inject_fault(s.ctx, B.RTE_FAULT_EXPIRE_WAIT)
    assert _status(s.forward, wl.groups, wl.n_steps) == TIMEOUT
    s.forward(wl.groups, wl.n_steps)
    curves = s.readout(wl.detectors).cpu().numpy()
    s.close()
    assert rel_l2(curves[0], _oracle_curves(wl)) < 1e-5


def test_timeout_word_is_per_context():
    """A timeout in one context leaves another context's march untouched."""
    from paper_2202_09421_gb300 import binding as B
    wl = _wl()
    s1, s2 = _tc_solver(wl), _tc_solver(wl)
    B.rte_inject_fault(s1.ctx, B.RTE_FAULT_TIMEOUT_WORD)
    s2.forward(wl.groups, wl.n_steps)
    curves = s2.readout(wl.detectors).cpu().numpy()
    assert _status(s1.forward, wl.groups, wl.n_steps) == TIMEOUT
    s1.close()
    s2.close()
    assert rel_l2(curves[0], _oracle_curves(wl)) < 1e-5


def test_fault_injection_rejected_where_there_are_no_device_waits():
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl = _wl()
    s = FCDOMSolver(wl.grid, wl.optics, _t(wl.mua), _t(wl.mus), wl.c, wl.dt)
    assert _status(B.rte_inject_fault, s.ctx, B.RTE_FAULT_TIMEOUT_WORD) == UNSUPPORTED
    s2 = _tc_solver(wl)
    assert _status(B.rte_inject_fault, s2.ctx, 9) == INVALID_ARG
    s.close()
    s2.close()
