"""GB300 (sm_103a) FC-DOM solver for the 2D time-domain radiative transfer
equation and its adjoint gradient (Gaggioli & Bruno, arXiv 2202.09421).

The compute path is the CUDA library built from csrc/ (C ABI in
include/rte.h); this package only marshals arguments to it."""
from .build import LIB, build  # noqa: F401


def __getattr__(name):
    # Loading the binding imports torch and opens the CUDA library; keep that
    # out of plain ``import paper_2202_09421_gb300`` (the build step needs it).
    if name in ("binding", "solver"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    if name in ("FCDOMSolver", "RTEObjective"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
