"""Host logic of the inverse solver (Algorithm 2) on CPU: the error measure
of eq. (errl2), the synthetic noise model, and the bound-constrained
L-BFGS-B loop driven by a quadratic objective whose minimiser is known."""
import numpy as np
import pytest

from paper_2202_09421_gb300.inverse import node_areas, reconstruct, relative_error
from rte_inputs import Grid, add_relative_noise, workload_inverse


def test_node_areas_integrate_the_domain():
    g = Grid(17, 11, 0.0, 2.0, -1.0, 0.5, 16)
    A = node_areas(g)
    assert A.shape == (11, 17)
    assert abs(A.sum() - 2.0 * 1.5) < 1e-12
    # trapezoid rule is exact for a bilinear function
    x = np.linspace(0.0, 2.0, 17)
    y = np.linspace(-1.0, 0.5, 11)
    f = (1 + x[None, :]) * (2 + y[:, None])
    exact = (2.0 + 2.0 ** 2 / 2) * ((2 * 0.5 + 0.5 ** 2 / 2) - (2 * -1 + 1 / 2))
    assert abs((A * f).sum() - exact) < 1e-12


def test_relative_error_closed_form():
    g = Grid(9, 9, 0.0, 1.0, 0.0, 1.0, 16)
    A = node_areas(g)
    a_t = np.full((9, 9), 2.0)
    assert relative_error(a_t, a_t, A) == 0.0
    assert abs(relative_error(a_t * 1.1, a_t, A) - 0.1) < 1e-12
    assert abs(relative_error(np.zeros_like(a_t), a_t, A) - 1.0) < 1e-12


def test_noise_model_is_seeded_and_relative():
    G = np.abs(np.random.default_rng(1).standard_normal((4, 32, 500))) + 1.0
    n1 = add_relative_noise(G, 0.1, seed=5)
    n2 = add_relative_noise(G, 0.1, seed=5)
    assert np.array_equal(n1, n2)
    rel = (n1 - G) / G
    assert abs(rel.mean()) < 3e-3 and abs(rel.std() - 0.1) < 3e-3
    assert not np.array_equal(n1, add_relative_noise(G, 0.1, seed=6))


def test_lbfgsb_loop_reaches_the_bounded_minimiser():
    """J(a) = 1/2 sum w (a - t)^2 with t partly outside [lo, hi]: the loop must
    return clip(t, lo, hi) and keep every iterate inside the bounds."""
    rng = np.random.default_rng(3)
    t = rng.uniform(0.0, 1.5, size=(12, 10))
    w = rng.uniform(0.5, 2.0, size=(12, 10))
    lo, hi = 0.1, 1.0
    seen = []

    def evaluate(a):
        seen.append(a.copy())
        d = a - t
        return 0.5 * float(np.sum(w * d * d)), w * d

    A = np.ones_like(t)
    out = reconstruct(evaluate, np.full_like(t, lo), lo, hi, max_iter=50, a_true=np.clip(t, lo, hi), area=A)
    assert np.allclose(out["a"], np.clip(t, lo, hi), atol=1e-6)
    assert all(x.min() >= lo - 1e-15 and x.max() <= hi + 1e-15 for x in seen)
    E = [h["E"] for h in out["history"]]
    assert E[-1] < 1e-5 < E[0]
    assert out["nfev"] == len(seen)                   # no point evaluated twice in a row


def test_inverse_workload_layouts():
    ts = workload_inverse("ts", n=64, n_steps=100)
    mss = workload_inverse("mss", n=64, n_steps=100)
    tgt = workload_inverse("ts", n=64, n_steps=100, target=True)
    assert len(ts.groups) == 16 and all(len(g) == 1 for g in ts.groups)
    assert len(mss.groups) == 4 and all(len(g) == 4 for g in mss.groups)
    # the same 16 beam positions in both modes; MSS delays within [0, T/2]
    pos = sorted((b.x, b.y) for g in ts.groups for b in g)
    assert pos == sorted((b.x, b.y) for g in mss.groups for b in g)
    assert all(0.0 <= b.tau <= 0.5 * 100 * 0.04 for g in mss.groups for b in g)
    assert np.all(ts.mua == 0.1) and tgt.mua.max() > 0.3 and tgt.mua.min() == 0.1
