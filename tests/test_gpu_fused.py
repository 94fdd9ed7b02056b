"""GPU parity of the tile-local fused step (rte_set_pass_variant 3: one
kernel per step over the subdomains of Sec. 4.4 / Algorithm 1, FP32) against
the oracle with the same decomposition, and against the two-pass kernels
applying the same decomposed operator; its checkpointed adjoint, CUDA-graph
replay and the fallback when the decomposition does not admit it."""
import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2
from oracle.rte import Solver
from rte_inputs import workload_custom

pytestmark = pytest.mark.gpu

FUSED = 3


def _solver(wl, parts, precision=0, ckpt=0, flags=0, variant=FUSED):
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    dev = torch.device("cuda:0")
    s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                    torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt, precision=precision,
                    fc_parts=parts, ckpt_interval=ckpt, flags=flags)
    B.rte_set_pass_variant(s.ctx, variant)
    return s


def _run(s, wl):
    fl = s.forward(wl.groups, wl.n_steps, list(wl.snap_steps))
    curves = s.readout(wl.detectors).cpu().numpy()
    states = np.stack([s.state(g).cpu().numpy() for g in range(len(wl.groups))])
    return fl.cpu().numpy(), curves, states


# (nx, ny, M, parts): owned ranges of 14..16 points, segments of 16..20;
# ragged partitions (46 = 15 + 15 + 16, 45 = 15 x 3) and both kernel forms.
CASES = [(48, 46, 16, (3, 3)), (64, 64, 32, (4, 4)), (45, 62, 32, (3, 4)), (64, 64, 16, (4, 4)), (96, 80, 32, (6, 5))]


@pytest.mark.parametrize("nx,ny,M,parts", CASES)
def test_fused_step_matches_oracle(nx, ny, M, parts):
    wl = workload_custom(nx, ny, M, 120, 0.04, L=(nx - 1) / 66, mus=20.0, n_groups=2, t_s=1.0, sigma_t=0.4)
    s = _solver(wl, parts)
    launches0 = s.kernel_launches()
    fl, curves, states = _run(s, wl)
    launches = s.kernel_launches() - launches0
    s.close()
    S = Solver(wl, fc_parts=parts)
    outs = [S.forward(g, wl.n_steps, wl.detectors, snap_steps=list(wl.snap_steps)) for g in wl.groups]
    c_ref = np.stack([o["curves"] for o in outs])
    f_ref = np.stack([[o["fluence"][k] for k in wl.snap_steps] for o in outs])
    u_ref = np.stack([np.moveaxis(o["u"], 0, -1) for o in outs])       # [g][j][i][m]
    ec, ef, eu = rel_l2(curves, c_ref), rel_l2(fl, f_ref), rel_l2(states, u_ref)
    print(f"fused {nx}x{ny} M{M} parts {parts}: curves {ec:.2e}, fluence {ef:.2e}, state {eu:.2e}; "
          f"{launches} launches")
    assert ec <= 1e-5 and ef <= 1e-5 and eu <= 1e-5
    # one kernel per step (plus fluence snapshots and the readout)
    assert launches <= wl.n_steps + len(wl.snap_steps) + 2


@pytest.mark.parametrize("precision", [0, 1])
def test_fused_step_matches_two_pass_decomposed(precision):
    """Same decomposed operator through the two-pass kernels (FP32 SIMT or
    3xTF32): the fused step agrees to FP32 rounding."""
    wl = workload_custom(64, 64, 32, 150, 0.04, L=63 / 66, mus=20.0, n_groups=2, t_s=1.0, sigma_t=0.4)
    s = _solver(wl, (4, 4), precision=precision)
    _, c_f, u_f = _run(s, wl)
    s.close()
    s = _solver(wl, (4, 4), precision=precision, variant=1)
    _, c_2, u_2 = _run(s, wl)
    s.close()
    print(f"prec {precision}: fused vs two-pass curves {rel_l2(c_f, c_2):.2e}, state {rel_l2(u_f, u_2):.2e}")
    assert rel_l2(c_f, c_2) <= 2e-6 and rel_l2(u_f, u_2) <= 2e-6


def test_fused_adjoint_gradient():
    """Checkpointed continuous adjoint with the fused step (recompute and
    adjoint march both fused) against the two-pass form of the same
    decomposed operator and against the oracle."""
    wl = workload_custom(48, 46, 16, 100, 0.04, L=47 / 66, mus=20.0, n_groups=2, t_s=1.0, sigma_t=0.4)
    tgt = workload_custom(48, 46, 16, 100, 0.04, L=47 / 66, mus=20.0, n_groups=2, t_s=1.0, sigma_t=0.4,
                          seed=7)
    meas = np.stack([Solver(tgt, fc_parts=(3, 3)).forward(g, 100, tgt.detectors)["curves"]
                     for g in tgt.groups]) * 0.8
    res = {}
    for variant in (FUSED, 1):
        s = _solver(wl, (3, 3), ckpt=13, variant=variant)
        s.forward(wl.groups, wl.n_steps)
        m = torch.tensor(meas, dtype=torch.float32, device=s.device)
        res[variant] = s.adjoint_gradient(wl.detectors, m)
        s.close()
    S = Solver(wl, fc_parts=(3, 3))
    Jo, gao = 0.0, 0.0
    for k, g in enumerate(wl.groups):
        j, a_, _, _ = S.adjoint_gradient(g, wl.n_steps, wl.detectors, meas[k])
        Jo, gao = Jo + j, gao + a_
    Jf, gaf, gbf = res[FUSED]
    J2, ga2, gb2 = res[1]
    print(f"fused adjoint: J {Jf:.6e} / {J2:.6e} / oracle {Jo:.6e}; grad_a vs two-pass "
          f"{rel_l2(gaf.cpu(), ga2.cpu()):.2e}, vs oracle {rel_l2(gaf.cpu(), gao):.2e}")
    assert abs(Jf - Jo) < 1e-5 * abs(Jo)
    assert rel_l2(gaf.cpu(), ga2.cpu()) < 1e-5 and rel_l2(gbf.cpu(), gb2.cpu()) < 1e-5
    assert rel_l2(gaf.cpu(), gao) < 1e-4


def test_fused_graph_replay_and_fallback():
    """CUDA-graph replay of the fused march equals the direct launches bit
    for bit (an odd step count leaves the state in the second buffer); a
    decomposition the fused step does not admit (owned ranges above 16)
    runs the two-pass kernels."""
    from paper_2202_09421_gb300 import binding as B
    wl = workload_custom(48, 46, 16, 37, 0.04, L=47 / 66, mus=20.0, n_groups=1, t_s=1.0, sigma_t=0.4)
    s = _solver(wl, (3, 3))
    _, c0, u0 = _run(s, wl)
    s.close()
    s = _solver(wl, (3, 3), flags=B.RTE_FLAG_CUDA_GRAPH)
    _run(s, wl)
    _, c1, u1 = _run(s, wl)
    assert s.graph_captures() == 1
    s.close()
    assert np.array_equal(c0, c1) and np.array_equal(u0, u1)
    # 48 / 2 = 24-point owned ranges: not admitted, same result as variant 1
    s = _solver(wl, (2, 2))
    n0 = s.kernel_launches()
    s.forward(wl.groups, wl.n_steps)
    assert s.kernel_launches() - n0 == 2 * wl.n_steps
    u_a = s.state(0).cpu().numpy()
    s.close()
    s = _solver(wl, (2, 2), variant=1)
    s.forward(wl.groups, wl.n_steps)
    u_b = s.state(0).cpu().numpy()
    s.close()
    assert np.array_equal(u_a, u_b)


# Tensor-core form (RTE_FLAG_TC_FUSED_STEP: 3xTF32, M = 32, every part
# owning 16 x 16 points).
TC_CASES = [(64, 64, (4, 4)), (96, 80, (6, 5))]


@pytest.mark.parametrize("nx,ny,parts", TC_CASES)
def test_fused_step_tensor_cores_matches_oracle(nx, ny, parts):
    """The tensor-core fused step against the oracle with the same
    decomposition (curves, fluence snapshots and the state of every group,
    beams on every face), and against the FP32 fused step."""
    wl = workload_custom(nx, ny, 32, 120, 0.04, L=(nx - 1) / 66, mus=20.0, n_groups=3, t_s=1.0, sigma_t=0.4)
    from paper_2202_09421_gb300 import binding as B
    s = _solver(wl, parts, precision=1, flags=B.RTE_FLAG_TC_FUSED_STEP)
    launches0 = s.kernel_launches()
    fl, curves, states = _run(s, wl)
    launches = s.kernel_launches() - launches0
    s.close()
    s = _solver(wl, parts, precision=0)
    fl0, curves0, states0 = _run(s, wl)
    s.close()
    S = Solver(wl, fc_parts=parts)
    outs = [S.forward(g, wl.n_steps, wl.detectors, snap_steps=list(wl.snap_steps)) for g in wl.groups]
    c_ref = np.stack([o["curves"] for o in outs])
    f_ref = np.stack([[o["fluence"][k] for k in wl.snap_steps] for o in outs])
    u_ref = np.stack([np.moveaxis(o["u"], 0, -1) for o in outs])
    ec, ef, eu = rel_l2(curves, c_ref), rel_l2(fl, f_ref), rel_l2(states, u_ref)
    d32 = rel_l2(states, states0)
    print(f"fused tc {nx}x{ny} parts {parts}: curves {ec:.2e}, fluence {ef:.2e}, state {eu:.2e}; "
          f"vs FP32 fused {d32:.2e}; {launches} launches")
    assert ec <= 1e-5 and ef <= 1e-5 and eu <= 1e-5
    assert d32 <= 2e-6 and rel_l2(curves, curves0) <= 2e-6
    # the per-node maximum error stays at FP32 level too
    assert np.max(np.abs(states - u_ref)) <= 1e-5 * np.max(np.abs(u_ref))
    assert launches <= wl.n_steps + len(wl.snap_steps) + 2


def test_fused_step_tensor_cores_adjoint_and_replay():
    """Checkpointed continuous adjoint through the tensor-core fused step
    (recompute and adjoint march) against the 3xTF32 two-pass form of the
    same decomposed operator and the oracle; CUDA-graph replay of the march
    equals the direct launches bit for bit."""
    from paper_2202_09421_gb300 import binding as B
    wl = workload_custom(64, 64, 32, 90, 0.04, L=63 / 66, mus=20.0, n_groups=2, t_s=1.0, sigma_t=0.4)
    tgt = workload_custom(64, 64, 32, 90, 0.04, L=63 / 66, mus=20.0, n_groups=2, t_s=1.0, sigma_t=0.4, seed=7)
    meas = np.stack([Solver(tgt, fc_parts=(4, 4)).forward(g, 90, tgt.detectors)["curves"]
                     for g in tgt.groups]) * 0.8
    res = {}
    for variant in (FUSED, 1):
        s = _solver(wl, (4, 4), precision=1, ckpt=11, variant=variant, flags=B.RTE_FLAG_TC_FUSED_STEP)
        s.forward(wl.groups, wl.n_steps)
        m = torch.tensor(meas, dtype=torch.float32, device=s.device)
        res[variant] = s.adjoint_gradient(wl.detectors, m)
        s.close()
    S = Solver(wl, fc_parts=(4, 4))
    Jo, gao = 0.0, 0.0
    for k, g in enumerate(wl.groups):
        j, a_, _, _ = S.adjoint_gradient(g, wl.n_steps, wl.detectors, meas[k])
        Jo, gao = Jo + j, gao + a_
    Jf, gaf, gbf = res[FUSED]
    J2, ga2, gb2 = res[1]
    print(f"fused tc adjoint: J {Jf:.6e} / {J2:.6e} / oracle {Jo:.6e}; grad_a vs two-pass "
          f"{rel_l2(gaf.cpu(), ga2.cpu()):.2e}, vs oracle {rel_l2(gaf.cpu(), gao):.2e}")
    assert abs(Jf - Jo) < 1e-5 * abs(Jo)
    assert rel_l2(gaf.cpu(), ga2.cpu()) < 1e-5 and rel_l2(gbf.cpu(), gb2.cpu()) < 1e-5
    assert rel_l2(gaf.cpu(), gao) < 1e-4

    wl = workload_custom(64, 64, 32, 37, 0.04, L=63 / 66, mus=20.0, n_groups=1, t_s=1.0, sigma_t=0.4)
    s = _solver(wl, (4, 4), precision=1, flags=B.RTE_FLAG_TC_FUSED_STEP)
    _, c0, u0 = _run(s, wl)
    s.close()
    s = _solver(wl, (4, 4), precision=1, flags=B.RTE_FLAG_CUDA_GRAPH | B.RTE_FLAG_TC_FUSED_STEP)
    _run(s, wl)
    _, c1, u1 = _run(s, wl)
    assert s.graph_captures() == 1
    s.close()
    assert np.array_equal(c0, c1) and np.array_equal(u0, u1)


def test_fused_step_tensor_cores_refused_outside_its_domain():
    """RTE_FLAG_TC_FUSED_STEP outside 3xTF32, M = 32 and 16-point parts is
    refused at creation."""
    from paper_2202_09421_gb300 import binding as B
    ok = workload_custom(64, 64, 32, 10, 0.04, L=63 / 66, mus=20.0, n_groups=1, t_s=1.0, sigma_t=0.4)
    ragged = workload_custom(48, 46, 32, 10, 0.04, L=47 / 66, mus=20.0, n_groups=1, t_s=1.0, sigma_t=0.4)
    m16 = workload_custom(64, 64, 16, 10, 0.04, L=63 / 66, mus=20.0, n_groups=1, t_s=1.0, sigma_t=0.4)
    for wl, parts, prec in ((ok, (4, 4), 0), (ok, (1, 1), 1), (ragged, (3, 3), 1), (m16, (4, 4), 1)):
        with pytest.raises(B.RTEError) as err:
            _solver(wl, parts, precision=prec, flags=B.RTE_FLAG_TC_FUSED_STEP)
        assert err.value.status == 7             # RTE_ERR_UNSUPPORTED
    _solver(ok, (4, 4), precision=1, flags=B.RTE_FLAG_TC_FUSED_STEP).close()


def test_fused_steps_tomo256_bench_configuration():
    """Both fused forms in the benchmark's launch configuration at full size:
    the 256 x 256, M = 32 tomography medium with 16 x 16 parts and all 16
    sources in one march (the FP32 form, and the tensor-core form with
    RTE_FLAG_TC_FUSED_STEP).  (1) Over the first 40 steps (the oracle's
    bounded sample) the first and the last source's curves, fluence and
    state match the oracle with the same decomposition.  (2) Over all 2000
    steps a source's curves equal a march of that source alone bit for bit
    (every subdomain's arithmetic is independent of the other sources in the
    launch), which holds at any size."""
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    from rte_inputs import workload_tomo256
    dev = torch.device("cuda:0")
    forms = {"fp32": (0, 0), "tensor cores": (1, B.RTE_FLAG_TC_FUSED_STEP)}

    def solver(wl, prec, flags):
        s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                        torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt, precision=prec,
                        fc_parts=(16, 16), flags=flags)
        B.rte_set_pass_variant(s.ctx, FUSED)
        return s

    short = workload_tomo256(n_steps=40)
    S = Solver(short, fc_parts=(16, 16))
    ends = (0, len(short.groups) - 1)
    ref = {gi: S.forward(short.groups[gi], short.n_steps, short.detectors, snap_steps=[39]) for gi in ends}
    for name, (prec, flags) in forms.items():
        s = solver(short, prec, flags)
        fl = s.forward(short.groups, short.n_steps, [39]).cpu().numpy()
        curves = s.readout(short.detectors).cpu().numpy()
        states = [s.state(gi).cpu().numpy() for gi in ends]
        s.close()
        for k, gi in enumerate(ends):
            o = ref[gi]
            ec, ef = rel_l2(curves[gi], o["curves"]), rel_l2(fl[gi][0], o["fluence"][39])
            eu = rel_l2(states[k], np.moveaxis(o["u"], 0, -1))
            print(f"fused {name}, tomo256 16x16 parts, 16 sources x 40, source {gi}: curves {ec:.2e}, "
                  f"fluence {ef:.2e}, state {eu:.2e}")
            assert ec <= 1e-5 and ef <= 1e-5 and eu <= 1e-5

    full = workload_tomo256()
    for name, (prec, flags) in forms.items():
        s = solver(full, prec, flags)
        s.forward(full.groups, full.n_steps)
        all_curves = s.readout(full.detectors).cpu().numpy()
        s.close()
        assert np.isfinite(all_curves).all() and all_curves.max() > 0
        for gi in (0, 9):
            s = solver(full, prec, flags)
            s.forward([full.groups[gi]], full.n_steps)
            alone = s.readout(full.detectors).cpu().numpy()[0]
            s.close()
            assert np.array_equal(alone, all_curves[gi]), (name, gi)
