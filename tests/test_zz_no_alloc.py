"""The allocation-free forward entry point, rte_forward_static.

Callers that cannot call cudaMalloc while they run (device memory already
held by another allocator, latency-critical loops where an allocation may
synchronise the device, a no-allocation policy after start-up) use it to
run a forward solve whose scratch lives in the library's static device
array.  This file is collected last so that a run stopping at its first
failure has already run every other test; it also passes on its own."""
import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2
from rte_inputs import workload_custom

pytestmark = pytest.mark.gpu
TOL = 1e-5      # the forward parity tolerance used by the other GPU tests
FP32, TF32X3 = 0, 1


def _solver(wl, **kw):
    from paper_2202_09421_gb300.solver import FCDOMSolver
    dev = torch.device("cuda:0")
    return FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                       torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt, **kw)


def _static_twice(s, wl, ref):
    from paper_2202_09421_gb300 import binding as B
    for call in range(2):
        out = torch.full((len(wl.groups), len(wl.detectors), wl.n_steps), float("nan"),
                         device="cuda:0", dtype=torch.float32)
        B.rte_forward_static(s.ctx, wl.groups, wl.n_steps, wl.detectors, out)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_l2(got, ref) <= TOL, (call, rel_l2(got, ref))


@pytest.mark.parametrize("precision", [FP32, TF32X3])
def test_static_forward_matches_allocating_path_twice(precision):
    """Two static calls in a row give the curves of rte_forward +
    rte_detector_readout on the same context, in the plain FP32 kernels and
    in the tensor-core (tcgen05, 3xTF32) passes."""
    wl = workload_custom(48, 40, 16, 90, 0.04, L=1.0, mus=20.0, n_groups=3, t_s=1.0, sigma_t=0.4)
    s = _solver(wl, precision=precision)
    s.forward(wl.groups, wl.n_steps)
    ref = s.readout(wl.detectors).cpu().numpy()
    assert np.abs(ref).max() > 0
    _static_twice(s, wl, ref)
    # the context's own forward results are untouched by the static calls
    again = s.readout(wl.detectors).cpu().numpy()
    assert np.array_equal(again, ref)
    s.close()


def test_static_forward_of_the_decomposed_operator_matches_the_fused_step():
    """With the subdomain decomposition and the tile-local fused step
    selected, rte_forward runs the fused step while the static call runs the
    two-pass kernels on the same operator: the curves agree to FP32 rounding."""
    from paper_2202_09421_gb300 import binding as B
    wl = workload_custom(48, 46, 16, 60, 0.04, L=47 / 66, mus=20.0, n_groups=2, t_s=1.0, sigma_t=0.4)
    s = _solver(wl, fc_parts=(3, 3))
    B.rte_set_pass_variant(s.ctx, 3)
    s.forward(wl.groups, wl.n_steps)
    ref = s.readout(wl.detectors).cpu().numpy()
    _static_twice(s, wl, ref)
    s.close()


def test_static_forward_reports_a_tensor_core_timeout():
    """The static call reads the context's timeout word like rte_forward."""
    from paper_2202_09421_gb300 import binding as B
    wl = workload_custom(48, 40, 16, 30, 0.04, L=1.0, mus=20.0, n_groups=1, t_s=1.0, sigma_t=0.4)
    s = _solver(wl, precision=TF32X3)
    out = torch.zeros((1, len(wl.detectors), wl.n_steps), device="cuda:0", dtype=torch.float32)
    B.rte_inject_fault(s.ctx, B.RTE_FAULT_TIMEOUT_WORD)
    with pytest.raises(B.RTEError) as err:
        B.rte_forward_static(s.ctx, wl.groups, wl.n_steps, wl.detectors, out)
    assert err.value.status == 5
    s.forward(wl.groups, wl.n_steps)
    ref = s.readout(wl.detectors).cpu().numpy()
    _static_twice(s, wl, ref)
    s.close()


def test_static_forward_rejects_oversize_and_short_outputs_before_device_work():
    from paper_2202_09421_gb300 import binding as B
    wl = workload_custom(256, 256, 32, 10, 0.01, L=4.0, n_groups=2)
    s = _solver(wl)
    out = torch.zeros((2, len(wl.detectors), 10), device="cuda:0", dtype=torch.float32)
    with pytest.raises(B.RTEError) as err:           # 2 groups x 5 x 8 MiB > 64 MiB
        B.rte_forward_static(s.ctx, wl.groups, 10, wl.detectors, out)
    assert err.value.status == 7
    short = torch.zeros((2, len(wl.detectors), 9), device="cuda:0", dtype=torch.float32)
    with pytest.raises(ValueError):
        B.rte_forward_static(s.ctx, wl.groups[:1], 10, wl.detectors, short[:1])
    s.close()
