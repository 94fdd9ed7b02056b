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


def test_static_forward_matches_allocating_path_twice():
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl = workload_custom(48, 40, 16, 90, 0.04, L=1.0, mus=20.0, n_groups=3, t_s=1.0, sigma_t=0.4)
    dev = torch.device("cuda:0")
    s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                    torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt)
    s.forward(wl.groups, wl.n_steps)
    ref = s.readout(wl.detectors).cpu().numpy()
    assert np.abs(ref).max() > 0
    for call in range(2):
        out = torch.full((len(wl.groups), len(wl.detectors), wl.n_steps), float("nan"),
                         device=dev, dtype=torch.float32)
        B.rte_forward_static(s.ctx, wl.groups, wl.n_steps, wl.detectors, out)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_l2(got, ref) <= TOL, (call, rel_l2(got, ref))
    # the context's own forward results are untouched by the static calls
    again = s.readout(wl.detectors).cpu().numpy()
    assert np.array_equal(again, ref)
    s.close()


def test_static_forward_rejects_oversize_before_device_work():
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl = workload_custom(256, 256, 32, 10, 0.01, L=4.0, n_groups=2)
    dev = torch.device("cuda:0")
    s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                    torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt)
    out = torch.zeros((2, len(wl.detectors), 10), device=dev, dtype=torch.float32)
    with pytest.raises(B.RTEError) as err:           # 2 groups x 5 x 8 MiB > 64 MiB
        B.rte_forward_static(s.ctx, wl.groups, 10, wl.detectors, out)
    assert err.value.status == 7
    s.close()
