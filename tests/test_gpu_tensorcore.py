"""GPU parity of the tcgen05 tensor-core forms of the FC operator products.

RTE_PREC_TF32X3 (split 3xTF32) must meet the FP32 tolerance of the forward
parity tests (relative L2 <= 1e-5 of fluence and detector curves against the
FP64 oracle); RTE_PREC_TF32 (one TF32 product) is the reduced-precision form,
held to its measured bound (<= 2e-2)."""
import numpy as np
import pytest
import torch

from gpu_helpers import gpu_forward, oracle_forward, rel_l2
from oracle.rte import Solver
from rte_inputs import workload_custom, workload_small, workload_tomo256

pytestmark = pytest.mark.gpu
TF32X3, TF32 = 1, 2


def _check(wl, label, precision, tol, flags=0):
    s, fl, curves = gpu_forward(wl, precision=precision, flags=flags)
    c_ref, f_ref, u_ref = oracle_forward(wl)
    ec, ef = rel_l2(curves, c_ref), rel_l2(fl, f_ref)
    print(f"{label} prec {precision}: curves rel L2 {ec:.3e}, fluence rel L2 {ef:.3e}")
    errs = []
    for g in range(len(wl.groups)):
        ug = s.state(g).cpu().numpy()
        uo = np.moveaxis(u_ref[g], 0, -1)
        errs.append(np.abs(ug - uo).max() / np.abs(uo).max())
    print(f"{label} prec {precision}: state max err / max {max(errs):.3e}")
    s.close()
    assert ec <= tol and ef <= tol, (ec, ef)
    return ec, ef


@pytest.mark.parametrize("precision,tol", [(TF32X3, 1e-5), (TF32, 2e-2)])
def test_tc_small64(precision, tol):
    _check(workload_small(n_steps=200, dt=0.05), "small64", precision, tol)


@pytest.mark.parametrize("nx,ny,M,groups", [(37, 53, 16, 3), (16, 16, 16, 1), (45, 29, 16, 2),
                                            (100, 70, 32, 2), (200, 131, 32, 1)])
def test_tc_ragged(nx, ny, M, groups):
    L = 1.0 if nx <= 100 else 3.0        # keep dx >= 1/66 cm so that dt = 0.04 ps is stable
    wl = workload_custom(nx, ny, M, 80, 0.04, L=L, mus=20.0, n_groups=groups, t_s=1.0, sigma_t=0.4)
    _check(wl, f"tc ragged{nx}x{ny}_M{M}", TF32X3, 1e-5)


@pytest.mark.parametrize("M", [16, 32])
def test_tc_scattering_contraction_form(M):
    """RTE_FLAG_TC_SCATTER: the scattering sum as a tcgen05 contraction into
    the x-pass accumulator meets the same FP32 tolerance."""
    wl = workload_custom(64, 48, M, 80, 0.04, L=1.0, mus=20.0, n_groups=2, t_s=1.0, sigma_t=0.4)
    _check(wl, f"tc-scatter M{M}", TF32X3, 1e-5, flags=1)


def test_tc_tomo256_truncated():
    wl = workload_tomo256(n_steps=60)
    wl.groups = wl.groups[:2]
    wl.snap_steps = [59]
    _check(wl, "tc tomo256x60", TF32X3, 1e-5)


def test_tc_adjoint_matches_oracle():
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl = workload_custom(48, 48, 16, 120, 0.04, L=1.0, mua=0.35, mus=8.0, n_groups=2,
                         heterogeneous=False, t_s=1.5, sigma_t=0.5)
    tgt = workload_custom(48, 48, 16, 120, 0.04, L=1.0, mua=0.35, mus=8.0, n_groups=2,
                          heterogeneous=True, t_s=1.5, sigma_t=0.5)
    St = Solver(tgt)
    meas = np.stack([St.forward(g, wl.n_steps, tgt.detectors)["curves"] for g in tgt.groups])
    dev = torch.device("cuda:0")
    s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                    torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt,
                    ckpt_interval=25, precision=TF32X3)
    s.forward(wl.groups, wl.n_steps)
    J, ga, gb = s.adjoint_gradient(wl.detectors, torch.tensor(meas, dtype=torch.float32, device=dev))
    S = Solver(wl)
    Jo, gao, gbo = 0.0, 0.0, 0.0
    for k, g in enumerate(wl.groups):
        j, a_, b_, _ = S.adjoint_gradient(g, wl.n_steps, wl.detectors, meas[k])
        Jo, gao, gbo = Jo + j, gao + a_, gbo + b_
    print(f"tc adjoint: J {J:.6e} vs {Jo:.6e}; grad_a {rel_l2(ga.cpu(), gao):.2e}; grad_b {rel_l2(gb.cpu(), gbo):.2e}")
    assert abs(J - Jo) < 1e-5 * abs(Jo)
    assert rel_l2(ga.cpu(), gao) < 1e-4 and rel_l2(gb.cpu(), gbo) < 1e-4
    s.close()


def test_tc_unsupported_sizes_are_rejected():
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    dev = torch.device("cuda:0")
    for nx, M in ((300, 16), (64, 24), (64, 8)):
        wl = workload_custom(nx, 64, M, 10, 0.01, L=1.0, n_groups=1)
        with pytest.raises(B.RTEError) as err:
            FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                        torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt,
                        precision=TF32X3)
        assert err.value.status == 7
