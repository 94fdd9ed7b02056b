"""Batched mixed-size forward (rte_forward_batch) and the CUDA-graph form of
the march (RTE_FLAG_CUDA_GRAPH).

A batched march advances every medium exactly as its own rte_forward would:
its curves and states must equal those of the single-medium call (same
kernel body and operation order), and the FP64 oracle within the FP32
tolerance.  The graph form replays the same launches: identical results,
one capture for repeated calls with the same sizes and buffers."""
import numpy as np
import pytest
import torch

from gpu_helpers import oracle_forward, rel_l2
from rte_inputs import workload_custom

pytestmark = pytest.mark.gpu
FP32, TF32X3, BF16X3 = 0, 1, 3
GRAPH = 2


def _solver(wl, precision, flags=0, ckpt=0):
    from paper_2202_09421_gb300.solver import FCDOMSolver
    dev = torch.device("cuda:0")
    return FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                       torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt,
                       ckpt_interval=ckpt, precision=precision, flags=flags)


def _media(M, sizes, n_steps=80, seed0=11):
    """Media of different grid sizes at equal spacing dx = 1/66 cm."""
    out = []
    for k, (nx, ny, G) in enumerate(sizes):
        out.append(workload_custom(nx, ny, M, n_steps, 0.04, L=(nx - 1) / 66.0, mus=20.0, n_groups=G,
                                   seed=seed0 + k, t_s=1.0, sigma_t=0.4))
    return out


def _run_single(wls, precision, flags=0, variant=1):
    """Single-medium runs, by default on the one-tile-per-CTA passes (the
    kernel body the batched launch shares)."""
    from paper_2202_09421_gb300 import binding as B
    res = []
    for wl in wls:
        s = _solver(wl, precision, flags)
        if precision != FP32:
            B.rte_set_pass_variant(s.ctx, variant)
        s.forward(wl.groups, wl.n_steps)
        res.append((s.readout(wl.detectors).cpu().numpy(),
                    [s.state(g).cpu().numpy() for g in range(len(wl.groups))]))
        s.close()
    return res


def _run_batch(wls, precision, flags=0, repeats=1):
    from paper_2202_09421_gb300.solver import forward_batch
    solvers = [_solver(wl, precision, flags) for wl in wls]
    for _ in range(repeats):
        forward_batch(solvers, [wl.groups for wl in wls], wls[0].n_steps)
    launches = solvers[0].kernel_launches()             # before the readout kernels
    res = [(s.readout(wl.detectors).cpu().numpy(), [s.state(g).cpu().numpy() for g in range(len(wl.groups))])
           for s, wl in zip(solvers, wls)]
    return solvers, res, launches


@pytest.mark.parametrize("precision,M,sizes", [
    (TF32X3, 16, [(48, 40, 2), (100, 70, 1), (64, 64, 1), (37, 53, 3)]),
    (TF32X3, 32, [(130, 100, 1), (40, 36, 2), (70, 66, 1)]),
    (BF16X3, 32, [(70, 66, 1), (130, 100, 1)]),
    (TF32X3, 64, [(48, 40, 1), (300, 40, 1)]),
    (FP32, 16, [(48, 40, 2), (100, 70, 1)]),
])
def test_batch_equals_single(precision, M, sizes):
    wls = _media(M, sizes)
    single = _run_single(wls, precision)
    solvers, batch, launches = _run_batch(wls, precision)
    for k, ((c1, u1), (c2, u2)) in enumerate(zip(single, batch)):
        ec = rel_l2(c2, c1)
        eu = max(float(np.abs(a - b).max() / max(np.abs(a).max(), 1e-30)) for a, b in zip(u1, u2))
        print(f"batch prec {precision} M{M} medium {k} {sizes[k]}: curves rel diff {ec:.2e}, state {eu:.2e}")
        assert ec <= 1e-6 and eu <= 1e-6
    if precision != BF16X3:
        for k, wl in enumerate(wls[:2]):
            c_ref, _, _ = oracle_forward(wl, snaps=[])
            e = rel_l2(batch[k][0], c_ref)
            print(f"batch prec {precision} M{M} medium {k} vs oracle: {e:.2e}")
            assert e <= 1e-5
    if precision != FP32:
        assert launches == 2 * wls[0].n_steps, launches      # one x-pass and one y-pass per step
    for s in solvers:
        s.close()


@pytest.mark.parametrize("precision", [FP32, TF32X3])
def test_graph_forward_replays(precision):
    wl = _media(16, [(64, 48, 2)], n_steps=60)[0]
    ref = _run_single([wl], precision, variant=1)[0]
    s = _solver(wl, precision, flags=GRAPH)
    for rep in range(3):
        s.forward(wl.groups, wl.n_steps)
        c = s.readout(wl.detectors).cpu().numpy()
        u = [s.state(g).cpu().numpy() for g in range(len(wl.groups))]
        assert np.array_equal(c, ref[0]) and all(np.array_equal(a, b) for a, b in zip(u, ref[1])), rep
    assert s.graph_captures() == 1
    per = s.kernel_launches()
    # a different step count re-captures
    s.forward(wl.groups, wl.n_steps - 6)
    assert s.graph_captures() == 2
    assert s.kernel_launches() > per
    s.close()


def test_graph_batch_replays():
    wls = _media(32, [(70, 66, 1), (40, 36, 2)], n_steps=50)
    s1, once, _ = _run_batch(wls, TF32X3)
    for s in s1:
        s.close()
    solvers, res, launches = _run_batch(wls, TF32X3, flags=GRAPH, repeats=3)
    for (c1, u1), (c2, u2) in zip(once, res):
        assert np.array_equal(c1, c2) and all(np.array_equal(a, b) for a, b in zip(u1, u2))
    assert solvers[0].graph_captures() == 1
    assert launches == 3 * 2 * wls[0].n_steps
    for s in solvers:
        s.close()


def test_batch_then_adjoint():
    """The checkpoints of a batched march serve rte_adjoint_gradient of each
    medium as those of its own rte_forward do."""
    from paper_2202_09421_gb300.solver import forward_batch
    wls = _media(16, [(48, 40, 1), (40, 48, 2)], n_steps=60)
    dev = torch.device("cuda:0")
    grads = []
    for mode in ("single", "batch"):
        solvers = [_solver(wl, TF32X3, ckpt=20) for wl in wls]
        if mode == "single":
            for s, wl in zip(solvers, wls):
                s.forward(wl.groups, wl.n_steps)
        else:
            forward_batch(solvers, [wl.groups for wl in wls], wls[0].n_steps)
        out = []
        for s, wl in zip(solvers, wls):
            meas = torch.zeros((len(wl.groups), len(wl.detectors), wl.n_steps), device=dev)
            J, ga, gb = s.adjoint_gradient(wl.detectors, meas)
            out.append((J, ga.cpu().numpy(), gb.cpu().numpy()))
            s.close()
        grads.append(out)
    for (J1, a1, b1), (J2, a2, b2) in zip(*grads):
        assert abs(J1 - J2) <= 1e-6 * abs(J1)
        assert rel_l2(a2, a1) <= 1e-6 and rel_l2(b2, b1) <= 1e-6


def test_batch_rejects_mixed_settings():
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import forward_batch
    wa = _media(16, [(48, 40, 1)])[0]
    wb = _media(32, [(48, 40, 1)])[0]
    sa, sb = _solver(wa, TF32X3), _solver(wb, TF32X3)
    with pytest.raises(B.RTEError) as err:
        forward_batch([sa, sb], [wa.groups, wb.groups], 10)
    assert err.value.status == 1
    with pytest.raises(B.RTEError) as err:
        forward_batch([sa, sa], [wa.groups, wa.groups], 10)
    assert err.value.status == 1
    sa.close(); sb.close()


@pytest.mark.parametrize("precision", [TF32X3, FP32])
def test_batched_adjoint_equals_each_medium_alone(precision):
    """rte_adjoint_gradient_batch after a batched march: every medium's J and
    gradients equal its own rte_adjoint_gradient (same kernel bodies and
    operation order, checkpoints of the same march), bit for bit; one
    medium's against the FP64 oracle's continuous adjoint."""
    from oracle.rte import Solver
    from paper_2202_09421_gb300.solver import adjoint_gradient_batch, forward_batch
    wls = _media(16, [(40, 36, 2), (48, 40, 1), (33, 35, 1)], n_steps=70)
    ss = [_solver(w, precision, ckpt=20) for w in wls]
    forward_batch(ss, [w.groups for w in wls], wls[0].n_steps)
    meas = [0.8 * s.readout(w.detectors) for s, w in zip(ss, wls)]
    got = adjoint_gradient_batch(ss, [w.detectors for w in wls], meas)
    for s, w, m, (J, ga, gb) in zip(ss, wls, meas, got):
        J1, ga1, gb1 = s.adjoint_gradient(w.detectors, m)
        assert J == J1
        assert torch.equal(ga, ga1) and torch.equal(gb, gb1)
        assert float(ga.abs().max()) > 0
    w, (J, ga, gb) = wls[1], got[1]
    S = Solver(w)
    mref = meas[1].double().cpu().numpy()
    Jo, gao, gbo = 0.0, 0.0, 0.0
    for k, g in enumerate(w.groups):
        j, a_, b_, _ = S.adjoint_gradient(g, w.n_steps, w.detectors, mref[k])
        Jo, gao, gbo = Jo + j, gao + a_, gbo + b_
    assert abs(J - Jo) < 1e-5 * abs(Jo)
    assert rel_l2(ga.cpu(), gao) < 1e-4 and rel_l2(gb.cpu(), gbo) < 1e-4
    for s in ss:
        s.close()


def test_batched_adjoint_rejects_mixed_step_counts():
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import adjoint_gradient_batch
    wls = _media(16, [(40, 36, 1), (33, 35, 1)], n_steps=40)
    ss = [_solver(w, TF32X3, ckpt=10) for w in wls]
    ss[0].forward(wls[0].groups, 40)
    ss[1].forward(wls[1].groups, 30)
    meas = [torch.zeros((len(w.groups), len(w.detectors), n), device="cuda:0") for w, n in zip(wls, (40, 30))]
    with pytest.raises(B.RTEError) as e:
        adjoint_gradient_batch(ss, [w.detectors for w in wls], meas)
    assert e.value.status == 1
    for s in ss:
        s.close()
