"""GPU parity of the tcgen05 tensor-core forms of the FC operator products.

RTE_PREC_TF32X3 (split 3xTF32) must meet the FP32 tolerance of the forward
parity tests (relative L2 <= 1e-5 of fluence and detector curves against the
FP64 oracle).  The reduced-precision forms are held to four times the
relative error of one operand product, the quantity that sets the error of
D u: with unit roundoff u_T = 2^-11 (tf32) and u_B = 2^-8 (bf16), one
product hi_x hi_y errs by about 2u (TF32: 2^-10 ~ 9.8e-4, BF16: 2^-7 ~
7.8e-3), the split three-product form by about 3u^2 (bf16x3: 3 * 2^-16 ~
4.6e-5).  Bounds: TF32 4e-3, bf16x3 2e-4, BF16 3e-2."""
import numpy as np
import pytest
import torch

from gpu_helpers import gpu_forward, oracle_forward, rel_l2
from oracle.rte import Solver
from rte_inputs import workload_custom, workload_precision512, workload_small, workload_tomo256

pytestmark = pytest.mark.gpu
TF32X3, TF32, BF16X3, BF16 = 1, 2, 3, 4
TOL = {TF32X3: 1e-5, TF32: 4e-3, BF16X3: 2e-4, BF16: 3e-2}


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


@pytest.mark.parametrize("precision", [TF32X3, TF32, BF16X3, BF16])
def test_tc_small64(precision):
    _check(workload_small(n_steps=200, dt=0.05), "small64", precision, TOL[precision])


@pytest.mark.parametrize("nx,ny,M,groups", [(37, 53, 16, 3), (16, 16, 16, 1), (45, 29, 16, 2),
                                            (100, 70, 32, 2), (200, 131, 32, 1)])
def test_tc_ragged(nx, ny, M, groups):
    L = 1.0 if nx <= 100 else 3.0        # keep dx >= 1/66 cm so that dt = 0.04 ps is stable
    wl = workload_custom(nx, ny, M, 80, 0.04, L=L, mus=20.0, n_groups=groups, t_s=1.0, sigma_t=0.4)
    _check(wl, f"tc ragged{nx}x{ny}_M{M}", TF32X3, 1e-5)


def _stable_custom(nx, ny, M, groups, n_steps=80):
    """dx = 1/66 cm whatever nx, so that dt = 0.04 ps is stable."""
    return workload_custom(nx, ny, M, n_steps, 0.04, L=(nx - 1) / 66.0, mus=20.0, n_groups=groups,
                           t_s=1.0, sigma_t=0.4)


@pytest.mark.parametrize("nx,ny,M", [(384, 24, 16), (24, 300, 16), (512, 20, 16), (20, 512, 16),
                                     (260, 130, 32)])
def test_tc_long_lines(nx, ny, M):
    """Lines longer than 256 positions: three or four 128-row accumulator
    tiles in the x-pass, the y-pass output positions issued as two MMAs of
    N <= 256 each."""
    _check(_stable_custom(nx, ny, M, 1), f"tc long{nx}x{ny}_M{M}", TF32X3, 1e-5)


@pytest.mark.parametrize("nx,ny,groups", [(48, 40, 2), (130, 70, 1), (300, 40, 1), (40, 260, 1)])
def test_tc_m64(nx, ny, groups):
    """64 ordinates: two grid rows (columns) per slab tile, the scattering sum
    over 64 ordinates in the x-pass epilogue."""
    _check(_stable_custom(nx, ny, 64, groups), f"tc M64 {nx}x{ny}", TF32X3, 1e-5)


@pytest.mark.parametrize("nx,ny,M,groups", [(45, 29, 16, 2), (100, 70, 32, 2), (130, 70, 64, 1),
                                            (24, 300, 16, 1)])
@pytest.mark.parametrize("precision", [BF16X3, BF16])
def test_tc_bf16_ragged(nx, ny, M, groups, precision):
    """kind::f16 with BF16 operands: K chunks of 64 positions, ragged in K and
    in the tiles."""
    _check(_stable_custom(nx, ny, M, groups), f"tc bf16 {nx}x{ny}_M{M}", precision, TOL[precision])


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
    """M outside {16, 32, 64}, and the tensor-core scattering flag with BF16
    operands or M = 64, give RTE_ERR_UNSUPPORTED at rte_init_medium."""
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    dev = torch.device("cuda:0")
    for nx, M, prec, flags in ((64, 24, TF32X3, 0), (64, 8, TF32X3, 0), (64, 40, BF16, 0),
                               (64, 64, TF32X3, 1), (64, 32, BF16X3, 1)):
        wl = workload_custom(nx, 64, M, 10, 0.01, L=1.0, n_groups=1)
        with pytest.raises(B.RTEError) as err:
            FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                        torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt,
                        precision=prec, flags=flags)
        assert err.value.status == 7


def test_precision512_all_forms():
    """The 512 x 512, M = 64, g = 0.8 smooth random medium at full spatial and
    angular size, 16 steps (the oracle's bounded sample): every precision
    form against the FP64 oracle, each within its bound."""
    wl = workload_precision512(n_steps=16)
    wl.snap_steps = [15]
    c_ref, f_ref, _ = oracle_forward(wl)
    rows = []
    for prec in (0, TF32X3, TF32, BF16X3, BF16):
        s, fl, curves = gpu_forward(wl, precision=prec)
        s.close()
        ec, ef = rel_l2(curves, c_ref), rel_l2(fl, f_ref)
        rows.append((prec, ec, ef))
        print(f"precision512x16 prec {prec}: curves rel L2 {ec:.3e}, fluence rel L2 {ef:.3e}")
    for prec, ec, ef in rows:
        tol = 1e-5 if prec == 0 else TOL[prec]
        assert ec <= tol and ef <= tol, (prec, ec, ef)


@pytest.mark.parametrize("nx,ny,M,groups", [(100, 70, 32, 2), (200, 131, 16, 1), (256, 256, 32, 3), (45, 29, 16, 5)])
@pytest.mark.parametrize("precision", [TF32X3, TF32, BF16X3, BF16])
def test_pass_variants_agree(nx, ny, M, groups, precision):
    """The persistent warp-specialised passes, the pipelined y-pass and the
    one-tile-per-CTA passes (default) perform the same products and the same
    per-node arithmetic;
    the y-pass epilogues may contract the AB4 sum differently, so the states
    agree to FP32 rounding (relative L2 <= 1e-6 for the split forms), and
    for the single-product forms, whose operand rounding turns such
    differences into tf32 / bf16 rounding steps, to a tenth of their bound."""
    from paper_2202_09421_gb300 import binding as B
    wl = _stable_custom(nx, ny, M, groups, n_steps=40)
    states = []
    for variant in (0, 1, 2):
        from paper_2202_09421_gb300.solver import FCDOMSolver
        dev = torch.device("cuda:0")
        s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                        torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt, precision=precision)
        B.rte_set_pass_variant(s.ctx, variant)
        s.forward(wl.groups, wl.n_steps)
        states.append([s.state(g).cpu().numpy() for g in range(groups)])
        s.close()
    tol = 1e-6 if precision in (TF32X3, BF16X3) else TOL[precision] / 10
    for other in (0, 2):
        for a_, b_ in zip(states[other], states[1]):
            d = float(np.abs(a_ - b_).max() / max(np.abs(b_).max(), 1e-30))
            e = rel_l2(a_, b_)
            print(f"variants {other} vs 1, {nx}x{ny} M{M} prec {precision}: rel L2 {e:.2e}, max rel diff {d:.2e}")
            assert e <= tol


@pytest.mark.parametrize("precision", [TF32X3, BF16X3])
def test_autotune_keeps_a_valid_configuration(precision):
    """rte_autotune times the admissible configurations and keeps the fastest;
    the forward it leaves behind still meets the precision's parity bound."""
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl = _stable_custom(100, 70, 32, 2)
    dev = torch.device("cuda:0")
    s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                    torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt, precision=precision)
    choice, ms = s.autotune(wl.groups, 12)
    print(f"autotune prec {precision}: choice {choice}, times {ms}")
    assert choice in ms and ms[choice] == min(ms.values())
    # choice = schedule + 6 * TC scattering (schedules 0, 1, 2, 4, 5); the
    # persistent warp-specialised schedule and the TMA-fed x-pass have no TC
    # scattering (schedule 5 with it keeps its TMA-fed y-pass), the BF16
    # kinds none at all and no TMA-fed passes
    expected = {0, 1, 2, 4, 5, 7, 8, 11} if precision == TF32X3 else {0, 1, 2}
    assert set(ms) == expected
    s.forward(wl.groups, wl.n_steps)
    curves = s.readout(wl.detectors).cpu().numpy()
    s.close()
    c_ref, _, _ = oracle_forward(wl, snaps=[])
    e = rel_l2(curves, c_ref)
    print(f"autotune prec {precision}: curves rel L2 {e:.2e}")
    assert e <= TOL[precision]


@pytest.mark.parametrize("nx,ny,M,groups,precision", [(48, 40, 64, 2, TF32X3), (37, 53, 16, 3, TF32X3),
                                                      (200, 131, 32, 1, TF32X3), (130, 70, 64, 1, BF16X3),
                                                      (16, 16, 16, 1, TF32X3), (70, 250, 32, 2, TF32)])
def test_pipelined_ypass_matches_oracle(nx, ny, M, groups, precision):
    """The pipelined y-pass schedule (rte_set_pass_variant 2) against the FP64
    oracle: ragged tiles, 8-row epilogue chunks ragged in y, boundary rows in
    any chunk, M up to 64."""
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl = _stable_custom(nx, ny, M, groups)
    dev = torch.device("cuda:0")
    s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                    torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt, precision=precision)
    B.rte_set_pass_variant(s.ctx, 2)
    fl = s.forward(wl.groups, wl.n_steps, list(wl.snap_steps))
    curves = s.readout(wl.detectors).cpu().numpy()
    s.close()
    c_ref, f_ref, _ = oracle_forward(wl)
    ec, ef = rel_l2(curves, c_ref), rel_l2(fl.cpu().numpy(), f_ref)
    print(f"pipelined y {nx}x{ny} M{M} prec {precision}: curves rel L2 {ec:.3e}, fluence rel L2 {ef:.3e}")
    assert ec <= TOL[precision] and ef <= TOL[precision]


@pytest.mark.parametrize("nx,ny,M,groups", [(256, 256, 32, 3), (100, 70, 32, 2), (200, 131, 16, 1),
                                            (45, 29, 16, 5), (256, 37, 16, 2), (37, 256, 32, 1)])
@pytest.mark.parametrize("precision", [TF32X3, TF32])
def test_tma_fed_passes_match_one_tile_bitwise(nx, ny, M, groups, precision):
    """Schedules 4 (TMA-fed x-pass) and 5 (TMA-fed x- and y-passes: raw slab
    by tensor copies, converter warps, persistent CTAs) issue the same
    splits, the same MMAs in the same order and the same epilogue arithmetic
    as the one-tile passes, so the states and the detector curves (from the
    y-pass's exitance) after a march are bit for bit the same; ragged sizes
    exercise the zero fill of the tensor copies past the last line and
    position, and the partial last tile of columns."""
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl = _stable_custom(nx, ny, M, groups, n_steps=30)
    dev = torch.device("cuda:0")
    states, curves = [], []
    for variant in (1, 4, 5):
        s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                        torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt, precision=precision)
        B.rte_set_pass_variant(s.ctx, variant)
        s.forward(wl.groups, wl.n_steps)
        states.append([s.state(g).cpu().numpy() for g in range(groups)])
        curves.append(s.readout(wl.detectors).cpu().numpy())
        s.close()
    for other in (1, 2):
        for a_, b_ in zip(states[0], states[other]):
            assert np.abs(a_).max() > 0
            assert np.array_equal(a_, b_)
        assert np.abs(curves[0]).max() > 0
        assert np.array_equal(curves[0], curves[other])


@pytest.mark.parametrize("variant", [4, 5])
def test_tma_fed_passes_match_oracle(variant):
    """Schedules 4 and 5 on a ragged multi-group case against the FP64 oracle
    (the forward parity bound of the FP32-level forms)."""
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl = _stable_custom(100, 70, 32, 2)
    dev = torch.device("cuda:0")
    s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                    torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt, precision=TF32X3)
    B.rte_set_pass_variant(s.ctx, variant)
    fl = s.forward(wl.groups, wl.n_steps, list(wl.snap_steps))
    curves = s.readout(wl.detectors).cpu().numpy()
    s.close()
    ref, f_ref, _ = oracle_forward(wl)
    assert rel_l2(curves, ref) <= 1e-5, rel_l2(curves, ref)
    assert rel_l2(fl.cpu().numpy(), f_ref) <= 1e-5


def test_tma_fed_ypass_adjoint_matches_one_tile_bitwise():
    """The continuous adjoint march injects the data residual on the boundary
    (the rho term of the y-pass epilogue) and recomputes the forward from
    checkpoints; under schedule 5 both run the TMA-fed passes, and J and the
    gradients equal the one-tile schedule's bit for bit."""
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    wl = _stable_custom(72, 64, 32, 2, n_steps=50)
    dev = torch.device("cuda:0")
    out = []
    for variant in (1, 5):
        s = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev),
                        torch.tensor(wl.mus, dtype=torch.float32, device=dev), wl.c, wl.dt, precision=TF32X3,
                        ckpt_interval=13)
        B.rte_set_pass_variant(s.ctx, variant)
        s.forward(wl.groups, wl.n_steps)
        meas = 0.7 * s.readout(wl.detectors)
        J, ga, gb = s.adjoint_gradient(wl.detectors, meas)
        out.append((J, ga.cpu().numpy(), gb.cpu().numpy()))
        s.close()
    assert out[0][0] == out[1][0] and out[0][0] > 0
    assert np.abs(out[0][1]).max() > 0
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
