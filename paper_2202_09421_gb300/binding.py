"""ctypes binding of the C ABI in include/rte.h.  Argument marshalling only:
every step of the method runs in the CUDA library.  Loading fails loudly when
the library has not been built (there is no fallback path).

The functions keep the C names (rte_init_medium, rte_forward, ...); tensors
are passed as device pointers and must be contiguous CUDA float32."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_longlong, c_void_p

import torch  # loads the shared CUDA runtime the library links against

from .build import LIB

RTE_PREC_FP32 = 0      # plain FP32 SIMT kernels
RTE_PREC_TF32X3 = 1    # tcgen05, split 3xTF32 operands (FP32-level accuracy)
RTE_PREC_TF32 = 2      # tcgen05, one TF32 product (reduced precision)
RTE_PREC_BF16X3 = 3    # tcgen05 kind::f16, BF16 operands split hi + lo (three products)
RTE_PREC_BF16 = 4      # tcgen05 kind::f16, one BF16 product
RTE_FLAG_TC_SCATTER = 1  # x-pass scattering as a tcgen05 contraction
RTE_FLAG_CUDA_GRAPH = 2  # forward march captured and replayed as a CUDA graph
RTE_FLAG_PHOTON_BALANCE = 4  # record the FP64 photon-balance terms of every step
RTE_FLAG_TC_FUSED_STEP = 8  # schedule 3's contractions on the tensor cores (3xTF32, M = 32, 16-point parts)


class RteGrid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("xmin", c_double), ("xmax", c_double),
                ("ymin", c_double), ("ymax", c_double), ("M", c_int)]


class RteOptics(ctypes.Structure):
    _fields_ = [("g", c_double), ("n_in", c_double), ("n_out", c_double),
                ("hg_exponent", c_double), ("c", c_double)]


class RteParams(ctypes.Structure):
    _fields_ = [("dt", c_double), ("filter_alpha", c_double), ("filter_beta", c_double),
                ("ckpt_interval", c_int), ("precision", c_int), ("flags", c_int),
                ("fc_parts_x", c_int), ("fc_parts_y", c_int)]


class RteBeam(ctypes.Structure):
    _fields_ = [("x", c_double), ("y", c_double), ("theta", c_double), ("sigma_x", c_double),
                ("sigma_theta", c_double), ("t_s", c_double), ("sigma_t", c_double),
                ("tau", c_double), ("amplitude", c_double), ("profile", c_int)]


class RteSourceGroup(ctypes.Structure):
    _fields_ = [("beams", POINTER(RteBeam)), ("n_beams", c_int)]


class RteDetector(ctypes.Structure):
    _fields_ = [("x", c_double), ("y", c_double), ("sigma_d", c_double)]


class RTEError(RuntimeError):
    def __init__(self, status: int, where: str):
        detail = ""
        if status in (3, 4):           # OOM, CUDA: name the underlying CUDA error
            detail = f", {library().rte_last_cuda_error().decode()}"
        super().__init__(f"{where}: status {status} ({rte_status_string(status)}{detail})")
        self.status = status


EXPORTS = ("rte_init_medium", "rte_set_medium", "rte_forward", "rte_detector_readout",
           "rte_objective", "rte_adjoint_gradient", "rte_get_state", "rte_kernel_launches",
           "rte_destroy", "rte_status_string", "rte_host_fc_operator", "rte_host_phase_matrix",
           "rte_set_kernel_timing", "rte_kernel_times", "rte_forward_static", "rte_forward_batch",
           "rte_graph_captures", "rte_set_pass_variant", "rte_last_cuda_error",
           "rte_autotune", "rte_host_fc_operator_parts", "rte_host_segment_images", "rte_discrete_adjoint_gradient",
           "rte_host_bc_transpose", "rte_inject_fault", "rte_photon_balance", "rte_adjoint_gradient_batch")

_lib = None


def library() -> ctypes.CDLL:
    """The loaded librte_fcdom.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"CUDA library {LIB} is missing: build it with "
                           "`python -m paper_2202_09421_gb300.build` (or __graft_entry__.build())")
    lib = ctypes.CDLL(LIB)
    P = c_void_p
    sig = {
        "rte_init_medium": [POINTER(c_void_p), POINTER(RteGrid), P, P, POINTER(RteOptics),
                            POINTER(RteParams), P],
        "rte_set_medium": [P, P, P],
        "rte_forward": [P, POINTER(RteSourceGroup), c_int, c_int, POINTER(c_int), c_int, P],
        "rte_detector_readout": [P, POINTER(RteDetector), c_int, P],
        "rte_objective": [P, POINTER(RteDetector), c_int, P, POINTER(c_double)],
        "rte_adjoint_gradient": [P, POINTER(RteDetector), c_int, P, POINTER(c_double), P, P],
        "rte_discrete_adjoint_gradient": [P, POINTER(RteDetector), c_int, P, POINTER(c_double), P, P],
        "rte_get_state": [P, c_int, P],
        "rte_kernel_launches": [P],
        "rte_destroy": [P],
        "rte_status_string": [c_int],
        "rte_host_fc_operator": [c_int, c_double, c_double, c_double, P],
        "rte_host_phase_matrix": [c_int, c_double, c_double, P],
        "rte_host_fc_operator_parts": [c_int, c_double, c_double, c_double, c_int, P],
        "rte_host_segment_images": [c_int, c_double, c_double, c_double, c_int, P],
        "rte_host_bc_transpose": [c_int, c_double, c_double, P, P],
        "rte_set_kernel_timing": [P, c_int],
        "rte_kernel_times": [P, POINTER(c_double), POINTER(c_longlong)],
        "rte_forward_static": [P, POINTER(RteSourceGroup), c_int, c_int, POINTER(RteDetector), c_int, P],
        "rte_forward_batch": [POINTER(c_void_p), c_int, POINTER(POINTER(RteSourceGroup)), POINTER(c_int), c_int],
        "rte_graph_captures": [P],
        "rte_set_pass_variant": [P, c_int],
        "rte_inject_fault": [P, c_int],
        "rte_photon_balance": [P, P],
        "rte_adjoint_gradient_batch": [POINTER(c_void_p), c_int, POINTER(POINTER(RteDetector)), POINTER(c_int),
                                       POINTER(c_void_p), POINTER(c_double), POINTER(c_void_p), POINTER(c_void_p)],
        "rte_last_cuda_error": [],
        "rte_autotune": [P, POINTER(RteSourceGroup), c_int, c_int, POINTER(c_int), POINTER(ctypes.c_float)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = c_int
    lib.rte_kernel_launches.restype = c_longlong
    lib.rte_graph_captures.restype = c_longlong
    lib.rte_status_string.restype = ctypes.c_char_p
    lib.rte_last_cuda_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def rte_status_string(status: int) -> str:
    return library().rte_status_string(int(status)).decode()


def _check(status: int, where: str):
    if status != 0:
        raise RTEError(status, where)


def _dev_ptr(t: torch.Tensor | None, name: str):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA float32 tensor")
    return c_void_p(t.data_ptr())


def _stream_handle(stream) -> c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return c_void_p(stream.cuda_stream)


def make_beams(beams):
    arr = (RteBeam * max(1, len(beams)))()
    for k, b in enumerate(beams):
        arr[k] = RteBeam(b.x, b.y, b.theta, b.sigma_x, b.sigma_theta, b.t_s, b.sigma_t,
                         getattr(b, "tau", 0.0), getattr(b, "amplitude", 1.0),
                         int(getattr(b, "profile", 0)))
    return arr


def make_detectors(dets):
    arr = (RteDetector * len(dets))()
    for k, d in enumerate(dets):
        arr[k] = RteDetector(d.x, d.y, d.sigma_d)
    return arr


# ---------------------------------------------------------------- C-named calls
def rte_init_medium(grid, mua: torch.Tensor, mus: torch.Tensor, optics, params, stream=None):
    """grid: object with nx, ny, xmin, xmax, ymin, ymax, M; optics: g, n_in,
    n_out, hg_exponent and c (cm/ps); params: RteParams.  Returns the context
    handle (c_void_p)."""
    ctx = c_void_p()
    g = RteGrid(grid.nx, grid.ny, grid.xmin, grid.xmax, grid.ymin, grid.ymax, grid.M)
    o = RteOptics(optics.g, optics.n_in, optics.n_out, optics.hg_exponent, optics.c)
    _check(library().rte_init_medium(ctypes.byref(ctx), ctypes.byref(g), _dev_ptr(mua, "mua"),
                                     _dev_ptr(mus, "mus"), ctypes.byref(o), ctypes.byref(params),
                                     _stream_handle(stream)), "rte_init_medium")
    return ctx


def rte_set_medium(ctx, mua, mus):
    _check(library().rte_set_medium(ctx, _dev_ptr(mua, "mua"), _dev_ptr(mus, "mus")), "rte_set_medium")


def rte_forward(ctx, groups, n_steps: int, snap_steps=(), fluence_out=None):
    """groups: list of lists of beam objects (one list per generalized source)."""
    beam_arrays = [make_beams(bl) for bl in groups]
    garr = (RteSourceGroup * len(groups))()
    for k, bl in enumerate(groups):
        garr[k] = RteSourceGroup(ctypes.cast(beam_arrays[k], POINTER(RteBeam)), len(bl))
    snaps = (c_int * max(1, len(snap_steps)))(*snap_steps)
    _check(library().rte_forward(ctx, garr, len(groups), int(n_steps), snaps, len(snap_steps),
                                 _dev_ptr(fluence_out, "fluence_out")), "rte_forward")


def rte_forward_batch(ctxs, groups_per_ctx, n_steps: int):
    """ctxs: list of context handles; groups_per_ctx: one list of groups (each
    a list of beams) per context."""
    n = len(ctxs)
    keep = []
    garrs = (POINTER(RteSourceGroup) * n)()
    ngr = (c_int * n)()
    for i, groups in enumerate(groups_per_ctx):
        beam_arrays = [make_beams(bl) for bl in groups]
        garr = (RteSourceGroup * len(groups))()
        for k, bl in enumerate(groups):
            garr[k] = RteSourceGroup(ctypes.cast(beam_arrays[k], POINTER(RteBeam)), len(bl))
        keep.append((beam_arrays, garr))
        garrs[i] = ctypes.cast(garr, POINTER(RteSourceGroup))
        ngr[i] = len(groups)
    carr = (c_void_p * n)(*[c.value for c in ctxs])
    _check(library().rte_forward_batch(carr, n, garrs, ngr, int(n_steps)), "rte_forward_batch")


def rte_adjoint_gradient_batch(ctxs, dets_per_ctx, measured_per_ctx, dJ_dmua=None, dJ_dmus=None):
    """Batched continuous adjoint over contexts that marched the same steps:
    J per context (list of float); the gradients are written into the given
    per-context device tensors (lists, entries may be None)."""
    n = len(ctxs)
    det_arrays = [make_detectors(d) for d in dets_per_ctx]
    darr = (POINTER(RteDetector) * n)(*[ctypes.cast(a, POINTER(RteDetector)) for a in det_arrays])
    ndet = (c_int * n)(*[len(d) for d in dets_per_ctx])
    meas = (c_void_p * n)(*[_dev_ptr(m, "measured").value for m in measured_per_ctx])
    J = (c_double * n)()

    def ptrs(lst, name):
        if lst is None:
            return None
        return (c_void_p * n)(*[(_dev_ptr(t, name).value if t is not None else None) for t in lst])
    ga, gb = ptrs(dJ_dmua, "dJ_dmua"), ptrs(dJ_dmus, "dJ_dmus")
    carr = (c_void_p * n)(*[c.value for c in ctxs])
    _check(library().rte_adjoint_gradient_batch(carr, n, darr, ndet, meas, J, ga, gb), "rte_adjoint_gradient_batch")
    return [J[k] for k in range(n)]


def rte_set_pass_variant(ctx, variant: int):
    _check(library().rte_set_pass_variant(ctx, int(variant)), "rte_set_pass_variant")


def rte_autotune(ctx, groups, n_trial_steps: int):
    """Returns (choice, {choice: ms}) of the configurations tried."""
    beam_arrays = [make_beams(bl) for bl in groups]
    garr = (RteSourceGroup * len(groups))()
    for k, bl in enumerate(groups):
        garr[k] = RteSourceGroup(ctypes.cast(beam_arrays[k], POINTER(RteBeam)), len(bl))
    choice = c_int()
    ms = (ctypes.c_float * 12)(*([-1.0] * 12))
    _check(library().rte_autotune(ctx, garr, len(groups), int(n_trial_steps), ctypes.byref(choice), ms),
           "rte_autotune")
    return choice.value, {k: ms[k] for k in range(12) if ms[k] >= 0.0}


def rte_graph_captures(ctx) -> int:
    return int(library().rte_graph_captures(ctx))


def rte_detector_readout(ctx, dets, curves_out):
    _check(library().rte_detector_readout(ctx, make_detectors(dets), len(dets),
                                          _dev_ptr(curves_out, "curves_out")), "rte_detector_readout")


def rte_objective(ctx, dets, measured) -> float:
    J = c_double()
    _check(library().rte_objective(ctx, make_detectors(dets), len(dets), _dev_ptr(measured, "measured"),
                                   ctypes.byref(J)), "rte_objective")
    return J.value


def rte_adjoint_gradient(ctx, dets, measured, dJ_dmua=None, dJ_dmus=None) -> float:
    J = c_double()
    _check(library().rte_adjoint_gradient(ctx, make_detectors(dets), len(dets),
                                          _dev_ptr(measured, "measured"), ctypes.byref(J),
                                          _dev_ptr(dJ_dmua, "dJ_dmua"), _dev_ptr(dJ_dmus, "dJ_dmus")),
           "rte_adjoint_gradient")
    return J.value


def rte_discrete_adjoint_gradient(ctx, dets, measured, dJ_dmua=None, dJ_dmus=None) -> float:
    J = c_double()
    _check(library().rte_discrete_adjoint_gradient(ctx, make_detectors(dets), len(dets),
                                                   _dev_ptr(measured, "measured"), ctypes.byref(J),
                                                   _dev_ptr(dJ_dmua, "dJ_dmua"), _dev_ptr(dJ_dmus, "dJ_dmus")),
           "rte_discrete_adjoint_gradient")
    return J.value


def rte_photon_balance(ctx, out):
    """Photon-balance terms of the last forward (device float64 [group][step][3]:
    photons int Phi / c, absorption int a Phi, net outward boundary flux)."""
    if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA float64 tensor")
    _check(library().rte_photon_balance(ctx, c_void_p(out.data_ptr())), "rte_photon_balance")


def rte_get_state(ctx, group: int, out):
    _check(library().rte_get_state(ctx, int(group), _dev_ptr(out, "out")), "rte_get_state")


def rte_kernel_launches(ctx) -> int:
    return int(library().rte_kernel_launches(ctx))


def rte_host_fc_operator_parts(n: int, h: float, parts: int, alpha: float = 2.0, beta: float = 55.0):
    """Host FP64 decomposed FC derivative operator (numpy n x n), Sec. 4.4."""
    import numpy as np
    out = np.zeros((n, n), dtype=np.float64)
    _check(library().rte_host_fc_operator_parts(n, h, alpha, beta, int(parts), c_void_p(out.ctypes.data)),
           "rte_host_fc_operator_parts")
    return out


def rte_host_segment_images(n: int, h: float, parts: int, alpha: float = 2.0, beta: float = 55.0):
    """The tensor-core fused step's segment-operator images (numpy float32
    [parts][2][16][32]: hi and lo tiles in the swizzled K-major order)."""
    import numpy as np
    out = np.zeros((parts, 2, 16, 32), dtype=np.float32)
    _check(library().rte_host_segment_images(n, h, alpha, beta, int(parts), c_void_p(out.ctypes.data)),
           "rte_host_segment_images")
    return out


def rte_host_fc_operator(n: int, h: float, alpha: float = 2.0, beta: float = 55.0):
    """Host FP64 FC derivative operator (numpy n x n)."""
    import numpy as np
    out = np.zeros((n, n), dtype=np.float64)
    _check(library().rte_host_fc_operator(n, h, alpha, beta, c_void_p(out.ctypes.data)),
           "rte_host_fc_operator")
    return out


def rte_host_phase_matrix(M: int, g: float, exponent: float = 1.5):
    import numpy as np
    out = np.zeros((M, M), dtype=np.float64)
    _check(library().rte_host_phase_matrix(M, g, exponent, c_void_p(out.ctypes.data)),
           "rte_host_phase_matrix")
    return out


def rte_host_bc_transpose(M: int, n_in: float = 1.4, n_out: float = 1.0):
    """(src [8][M][4] int, f [8][M][4] float64): the transposed boundary map."""
    import numpy as np
    src = np.zeros((8, M, 4), dtype=np.int32)
    f = np.zeros((8, M, 4), dtype=np.float64)
    _check(library().rte_host_bc_transpose(M, n_in, n_out, c_void_p(src.ctypes.data), c_void_p(f.ctypes.data)),
           "rte_host_bc_transpose")
    return src, f


def rte_set_kernel_timing(ctx, on: bool):
    _check(library().rte_set_kernel_timing(ctx, int(bool(on))), "rte_set_kernel_timing")


def rte_kernel_times(ctx):
    """(ms per pass [x, y], launches per pass [x, y]) since the last call."""
    ms = (c_double * 2)()
    cnt = (c_longlong * 2)()
    _check(library().rte_kernel_times(ctx, ms, cnt), "rte_kernel_times")
    return [ms[0], ms[1]], [cnt[0], cnt[1]]


def rte_forward_static(ctx, groups, n_steps: int, dets, curves_out):
    """Forward solve and detector curves without any device allocation: all
    per-call scratch sits in the library's 64 MiB static device array (for
    callers that cannot call cudaMalloc while they run; see include/rte.h)."""
    need = len(groups) * len(dets) * int(n_steps)
    if curves_out.numel() < need:
        raise ValueError(f"curves_out holds {curves_out.numel()} floats; [group][det][step] needs {need}")
    beam_arrays = [make_beams(bl) for bl in groups]
    garr = (RteSourceGroup * len(groups))()
    for k, bl in enumerate(groups):
        garr[k] = RteSourceGroup(ctypes.cast(beam_arrays[k], POINTER(RteBeam)), len(bl))
    _check(library().rte_forward_static(ctx, garr, len(groups), int(n_steps), make_detectors(dets),
                                        len(dets), _dev_ptr(curves_out, "curves_out")),
           "rte_forward_static")


RTE_FAULT_CLEAR, RTE_FAULT_TIMEOUT_WORD, RTE_FAULT_EXPIRE_WAIT = 0, 1, 2


def rte_inject_fault(ctx, kind: int):
    """Host-side failure injection for tests of the timeout path (see
    include/rte.h): set the context's timeout word, or make the next march's
    first tensor-core pass run one bounded wait out."""
    _check(library().rte_inject_fault(ctx, int(kind)), "rte_inject_fault")


def rte_destroy(ctx):
    _check(library().rte_destroy(ctx), "rte_destroy")
