"""CPU tests of the C-ABI library: it loads, exports every symbol that
include/rte.h declares, its host FP64 set-up matches the oracle's operators
(separately written code, same recipe), and argument validation returns
error codes before any device work."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "rte.h")


@pytest.fixture(scope="module")
def B():
    from paper_2202_09421_gb300 import build
    build(force=False)
    from paper_2202_09421_gb300 import binding
    binding.library()
    return binding


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:rte_status|const char\*|long long)\s+(rte_\w+)\(", text, re.M)))


def test_header_declares_the_boundary_calls():
    syms = declared_symbols()
    for name in ("rte_init_medium", "rte_forward", "rte_adjoint_gradient", "rte_detector_readout",
                 "rte_destroy", "rte_status_string"):
        assert name in syms


def test_library_exports_every_declared_symbol(B):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(rte_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    assert set(B.EXPORTS) == set(declared_symbols())


@pytest.mark.parametrize("n,h", [(16, 0.1), (61, 0.1), (64, 2 / 63), (256, 4 / 255), (37, 0.03), (512, 4 / 511)])
def test_host_fc_operator_matches_oracle(B, n, h):
    """Separately built tables and operator (library: Lagrange-basis normal
    equations, circulant kernel in closed form; oracle: Gram basis, QR, FFT)
    agree to ~1e-12 relative."""
    from oracle import fcgram
    D = B.rte_host_fc_operator(n, h)
    Do = fcgram.derivative_matrix(n, h)
    assert np.abs(D - Do).max() < 1e-12 * np.abs(Do).max()


@pytest.mark.parametrize("M,g,e", [(8, 0.0, 1.5), (16, 0.9, 1.5), (32, 0.8, 1.0), (64, 0.9, 1.5)])
def test_host_phase_matrix_matches_oracle(B, M, g, e):
    from oracle import rte
    assert np.abs(B.rte_host_phase_matrix(M, g, e) - rte.phase_matrix(M, g, e)).max() < 1e-14


def test_fc_tables_generators_agree():
    """The library's table header and the oracle's table file come from two
    independent generators of the same recipe; they agree to FP64 rounding."""
    from oracle import fcgram
    Q, A = fcgram.load_tables()
    txt = open(os.path.join(ROOT, "paper_2202_09421_gb300", "csrc", "fcgram_table.h")).read()
    body = txt.split("= {", 1)[1]
    vals = np.array([float(v) for v in re.findall(r"[-+]?\d+\.\d*(?:e[-+]?\d+)?", body)]).reshape(25, 5)
    comb = A @ Q.T
    assert np.abs(vals - comb).max() < 1e-14 * np.abs(comb).max()


def test_argument_validation_without_device(B):
    """Bad sizes and pointers are rejected before any CUDA call."""
    lib = B.library()
    ctx = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    o = B.RteOptics(0.9, 1.4, 1.0, 1.5, 0.0214)
    p = B.RteParams(0.05, 2.0, 55.0, 0, 0)
    bad_grids = [B.RteGrid(8, 64, 0, 1, 0, 1, 16),       # nx too small
                 B.RteGrid(64, 64, 0, 1, 0, 1, 12),      # M not a multiple of 8
                 B.RteGrid(64, 64, 1, 0, 0, 1, 16)]      # xmax < xmin
    for g in bad_grids:
        assert lib.rte_init_medium(ctypes.byref(ctx), ctypes.byref(g), dummy, dummy, ctypes.byref(o),
                                   ctypes.byref(p), None) == 1
    big = B.RteGrid(1024, 64, 0, 1, 0, 1, 16)
    assert lib.rte_init_medium(ctypes.byref(ctx), ctypes.byref(big), dummy, dummy, ctypes.byref(o),
                               ctypes.byref(p), None) == 7
    g = B.RteGrid(64, 64, 0, 1, 0, 1, 16)
    assert lib.rte_init_medium(ctypes.byref(ctx), ctypes.byref(g), None, dummy, ctypes.byref(o),
                               ctypes.byref(p), None) == 1
    neg_dt = B.RteParams(-0.1, 2.0, 55.0, 0, 0)
    assert lib.rte_init_medium(ctypes.byref(ctx), ctypes.byref(g), dummy, dummy, ctypes.byref(o),
                               ctypes.byref(neg_dt), None) == 1
    assert lib.rte_forward(None, None, 0, 0, None, 0, None) == 1
    assert lib.rte_destroy(None) == 1
    assert B.rte_status_string(2).startswith("dt outside")


@pytest.mark.parametrize("n,h,parts", [(64, 0.05, 2), (97, 0.02, 3), (256, 4 / 255, 4), (200, 0.03, 5)])
def test_host_decomposed_operator_matches_oracle(B, n, h, parts):
    """The library's decomposed operator (Sec. 4.4, built from its own
    FC-Gram table and closed-form kernel) against the oracle's per-segment
    FFT derivative applied to the identity."""
    from oracle.fcgram import fc_derivative_parts
    D = B.rte_host_fc_operator_parts(n, h, parts)
    Do = fc_derivative_parts(np.eye(n), h, axis=-1, parts=parts).T
    scale = np.abs(Do).max()
    # Segments of 34-66 points: the two FP64 routes (closed-form kernel sums
    # against FFT) already differ by 1.04e-12 relative on a global line of 34
    # points, the level of these short lines.
    assert np.abs(D - Do).max() <= 4e-12 * scale
    # block structure: row i has support only in its owner's segment
    from oracle.fcgram import subdomain_segments
    for lo, hi, slo, shi in subdomain_segments(n, parts):
        assert np.all(D[lo:hi, :slo] == 0) and np.all(D[lo:hi, shi:] == 0)


def test_host_decomposed_operator_rejects_short_segments(B):
    with pytest.raises(B.RTEError) as err:
        B.rte_host_fc_operator_parts(40, 0.05, 4)      # owned ranges of 10 -> segments of 12-14 points
    assert err.value.status == 1


@pytest.mark.parametrize("M", [8, 16, 32])
def test_host_bc_transpose_matches_oracle(B, M):
    """The library's transposed boundary table (what the discrete adjoint
    gathers through) against the oracle's transposed boundary map, pinned by
    the dot-product identity: at every boundary node of a grid, on a random
    field."""
    from oracle.rte import Solver
    from rte_inputs import workload_custom
    wl = workload_custom(16, 18, M, 4, 0.04)
    src, f = B.rte_host_bc_transpose(M, wl.optics.n_in, wl.optics.n_out)
    ubar = np.random.default_rng(M).standard_normal((M, wl.grid.ny, wl.grid.nx))
    ref = Solver(wl).bc_transpose(ubar)
    nx, ny = wl.grid.nx, wl.grid.ny
    worst = 0.0
    for j in range(ny):
        for i in range(nx):
            lf, rt, bt, tp = i == 0, i == nx - 1, j == 0, j == ny - 1
            if not (lf or rt or bt or tp):
                continue
            t = 4 + rt + 2 * tp if (lf or rt) and (bt or tp) else (0 if lf else 1 if rt else 2 if bt else 3)
            w = (f[t] * ubar[src[t], j, i]).sum(axis=1)
            worst = max(worst, np.abs(w - ref[:, j, i]).max())
    assert worst < 1e-13, worst


def test_header_is_plain_c():
    """include/rte.h is a C ABI: it compiles as C99 (and as C++) with no
    other header of this project and no torch or CUDA types."""
    import shutil
    import subprocess
    hdr = os.path.join(ROOT, "include", "rte.h")
    for compiler, lang, std in (("gcc", "c", "-std=c99"), ("g++", "c++", "-std=c++17")):
        if shutil.which(compiler) is None:
            pytest.skip(f"{compiler} not available")
        out = subprocess.run([compiler, "-fsyntax-only", "-x", lang, std, "-Wall", "-Wextra", "-Werror", hdr],
                             capture_output=True, text=True)
        assert out.returncode == 0, out.stderr
    includes = [ln for ln in open(hdr) if ln.lstrip().startswith("#include")]
    assert all("<stddef.h>" in ln or "<stdint.h>" in ln for ln in includes), includes


def test_binding_constants_match_the_header():
    """Every integer constant the header defines (#define RTE_..., and the
    rte_status codes) has the same value in the binding wherever the binding
    names it; the precisions and flags must all be there."""
    from paper_2202_09421_gb300 import binding
    text = open(HEADER).read()
    consts = {k: int(v) for k, v in re.findall(r"^#define\s+(RTE_\w+)\s+(\d+)\s*$", text, re.M)}
    consts.update({k: int(v) for k, v in re.findall(r"^\s*(RTE_\w+)\s*=\s*(\d+)\s*,?", text, re.M)})
    assert consts, "no constants parsed from the header"
    for name, value in consts.items():
        if hasattr(binding, name):
            assert getattr(binding, name) == value, name
    for name in consts:
        if name.startswith(("RTE_PREC_", "RTE_FLAG_")):
            assert hasattr(binding, name), name


@pytest.mark.parametrize("n,parts", [(64, 4), (96, 6), (256, 16)])
def test_host_segment_images_encode_the_decomposed_operator(B, n, parts):
    """The segment-operator images of the tensor-core fused step, decoded
    with the K-major 128-byte-swizzle layout of a tcgen05 operand (16-byte
    group p/4 of row i stored at group (p/4) xor (i mod 8)): hi is a tf32
    value (low 13 bits zero), hi + lo equals the decomposed operator's row of
    owned point lo + i at grid point lo - 2 + p to the split's rounding, and
    every entry outside the part's segment is zero."""
    from oracle.fcgram import subdomain_segments
    h = 1.0 / (n - 1)
    D = B.rte_host_fc_operator_parts(n, h, parts)
    img = B.rte_host_segment_images(n, h, parts)
    scale = np.abs(D).max()
    i_idx = np.arange(16)[:, None]
    p_idx = np.arange(32)[None, :]
    pos = ((p_idx >> 2) ^ (i_idx & 7)) * 4 + (p_idx & 3)          # [16][32] storage column
    for k, (lo, hi, slo, shi) in enumerate(subdomain_segments(n, parts)):
        hi_v = np.take_along_axis(img[k, 0], pos, axis=1).astype(np.float64)
        lo_v = np.take_along_axis(img[k, 1], pos, axis=1).astype(np.float64)
        assert np.all(img[k, 0].view(np.uint32) & 0x1FFF == 0)     # tf32-representable
        want = np.zeros((16, 32))
        for i in range(hi - lo):
            for p in range(32):
                x = lo - 2 + p
                if slo <= x < shi:
                    want[i, p] = D[lo + i, x]
        assert np.all((hi_v + lo_v)[want == 0] == 0)
        assert np.abs(hi_v + lo_v - want).max() <= 2.0 ** -21 * scale
        assert np.abs(hi_v - want).max() > 0 or np.abs(want).max() == 0   # lo carries the rest


def test_host_segment_images_rejects_long_parts(B):
    """Parts owning more than 16 points have no image (the fused step
    does not take them)."""
    with pytest.raises(B.RTEError):
        B.rte_host_segment_images(96, 1.0 / 95, 3)
