"""Pins of the oracle's continuous adjoint gradient (Sec. 3.4-3.6) against
finite differences of its own forward solve (Sec. 3.5 protocol: direction
delta a = 1 and per-node Kronecker directions; central differences).

The paper's adjoint is continuous (differentiate, then discretise), so the
agreement is at discretisation level and improves under refinement (Table 1
reports 8e-5 .. 9.7e-4 at N = 200, M = 32, 60000 steps)."""
import numpy as np
import pytest

from oracle.rte import Solver
from rte_inputs import workload_custom


def _case(n, steps, dt, heterogeneous):
    return workload_custom(n, n, 8, steps, dt, L=1.0, g=0.9, mua=0.35, mus=8.0,
                           heterogeneous=heterogeneous, t_s=3.0, sigma_t=1.0)


def _objective(n, steps, dt, a, b, measured):
    wl = _case(n, steps, dt, False)
    wl.mua, wl.mus = a, b
    S = Solver(wl)
    return S.objective(S.forward(wl.groups[0], steps, wl.detectors)["curves"], measured)


@pytest.fixture(scope="module")
def gradients():
    out = {}
    for n, steps, dt in ((32, 1500, 0.04), (48, 2000, 0.03)):
        target = _case(n, steps, dt, True)
        St = Solver(target)
        measured = St.forward(target.groups[0], steps, target.detectors)["curves"]
        wl = _case(n, steps, dt, False)
        J, ga, gb, _ = Solver(wl).adjoint_gradient(wl.groups[0], steps, wl.detectors, measured)
        out[n] = dict(J=J, ga=ga, gb=gb, wl=wl, measured=measured, steps=steps, dt=dt)
    return out


def _fd(case, da=None, db=None, eps=1e-4):
    wl = case["wl"]
    n, steps, dt, meas = wl.grid.nx, case["steps"], case["dt"], case["measured"]
    da = np.zeros_like(wl.mua) if da is None else da
    db = np.zeros_like(wl.mus) if db is None else db
    Jp = _objective(n, steps, dt, wl.mua + eps * da, wl.mus + eps * db, meas)
    Jm = _objective(n, steps, dt, wl.mua - eps * da, wl.mus - eps * db, meas)
    return (Jp - Jm) / (2 * eps)


def test_adjoint_mua_uniform_direction_converges(gradients):
    """eq. (Errgrad) with delta a = 1: relative error below 5% at 32^2 and
    below 1.5% at 48^2, decreasing under refinement."""
    errs = []
    for n in (32, 48):
        c = gradients[n]
        adj = c["ga"].sum()
        fd = _fd(c, da=np.ones_like(c["ga"]))
        errs.append(abs(adj - fd) / abs(adj))
    assert errs[0] < 0.05 and errs[1] < 0.015 and errs[1] < errs[0], errs


def test_adjoint_mua_per_node(gradients):
    """eq. (FDwin22): per-node gradient against a Kronecker perturbation at
    the two nodes with the largest |dJ/da| at least 0.25 cm inside."""
    c = gradients[32]
    ga = c["ga"].copy()
    inner = np.zeros_like(ga, dtype=bool)
    inner[8:-8, 8:-8] = True                      # >= 0.25 cm from the boundary
    order = np.argsort(np.where(inner, np.abs(ga), 0).ravel())[::-1][:2]
    for flat in order:
        j, i = np.unravel_index(flat, ga.shape)
        da = np.zeros_like(ga)
        da[j, i] = 1.0
        fd = _fd(c, da=da)
        assert abs(ga[j, i] - fd) < 0.05 * abs(fd), (j, i, ga[j, i], fd)


def test_adjoint_mus_uniform_direction(gradients):
    """Extension to the scattering coefficient: dJ/db = -<lambda, u - P u>,
    checked along delta b = 1."""
    c = gradients[32]
    fd = _fd(c, db=np.ones_like(c["gb"]), eps=1e-3)
    adj = c["gb"].sum()
    assert abs(adj - fd) < 0.05 * abs(adj), (adj, fd)


def test_discrete_adjoint_against_the_continuous_one(gradients):
    """The exact discrete adjoint (the transpose of the march) on the same
    case: it matches central differences of the discrete objective along
    delta a = 1 and delta b = 1 to their truncation error, where the
    continuous adjoint is off by its discretisation error (3% here); the
    two gradients agree to that level away from the boundary."""
    c = gradients[32]
    wl = c["wl"]
    _, ga, gb = Solver(wl).discrete_adjoint_gradient(wl.groups[0], c["steps"], wl.detectors, c["measured"])
    fd_a = _fd(c, da=np.ones_like(ga))
    fd_b = _fd(c, db=np.ones_like(gb), eps=1e-2)
    ea, eb = abs(ga.sum() - fd_a) / abs(fd_a), abs(gb.sum() - fd_b) / abs(fd_b)
    ca, cb = abs(c["ga"].sum() - fd_a) / abs(fd_a), abs(c["gb"].sum() - fd_b) / abs(fd_b)
    inner = np.zeros_like(ga, dtype=bool)
    inner[8:-8, 8:-8] = True
    d_inner = np.linalg.norm((ga - c["ga"])[inner]) / np.linalg.norm(ga[inner])
    print(f"delta a = 1: discrete {ea:.1e}, continuous {ca:.1e}; delta b = 1: discrete {eb:.1e}, "
          f"continuous {cb:.1e}; interior difference {d_inner:.1e}")
    assert ea < 1e-6 and eb < 1e-6
    assert ca > 100 * ea and cb > 100 * eb
    assert d_inner < 0.05


def test_adjoint_mss_group_uniform_direction():
    """The same protocol (delta a = 1, central differences) for a generalized
    source: four beams, one per face, fired with staggered delays as one MSS
    group (Sec. 2.2, eq. RTEsources2 summed over the group).  The continuous
    adjoint agrees to discretisation level (under 5 % at 32^2, as for a
    single beam), the exact discrete adjoint to the differences' truncation."""
    import dataclasses
    n, steps, dt = 32, 1500, 0.04
    base = workload_custom(n, n, 8, steps, dt, L=1.0, g=0.9, mua=0.35, mus=8.0, heterogeneous=False,
                           t_s=3.0, sigma_t=1.0, n_groups=4)
    beams = [dataclasses.replace(g[0], tau=1.5 * k) for k, g in enumerate(base.groups)]
    wl = dataclasses.replace(base, groups=[beams])
    tgt = dataclasses.replace(_case(n, steps, dt, True), groups=[beams])
    measured = Solver(tgt).forward(beams, steps, tgt.detectors)["curves"]
    S = Solver(wl)
    _, ga, _, _ = S.adjoint_gradient(beams, steps, wl.detectors, measured)
    _, gd, _ = S.discrete_adjoint_gradient(beams, steps, wl.detectors, measured)

    def J(a):
        Sp = Solver(dataclasses.replace(wl, mua=a))
        return Sp.objective(Sp.forward(beams, steps, wl.detectors)["curves"], measured)

    eps = 1e-4
    fd = (J(wl.mua + eps) - J(wl.mua - eps)) / (2 * eps)
    ec, ed = abs(ga.sum() - fd) / abs(fd), abs(gd.sum() - fd) / abs(fd)
    print(f"MSS group, delta a = 1: continuous {ec:.1e}, discrete {ed:.1e}")
    assert ec < 0.05 and ed < 1e-6
