"""Pins of the oracle's exact discrete adjoint (the reverse sweep of the
discrete march): it is the transpose of the tangent-linear march, so
<dJ/da, da> + <dJ/db, db> equals the forward-mode derivative to rounding,
and it is the gradient of the discrete objective, so central differences
agree to their truncation error.  The continuous adjoint of Sec. 3 only
reaches these to discretisation level (its own pins are in
test_oracle_adjoint.py)."""
import dataclasses

import numpy as np
import pytest

from oracle.rte import Solver
from rte_inputs import workload_custom


def _case(parts=(1, 1), groups=2):
    wl = workload_custom(22, 20, 8, 40, 0.04, L=21 / 66, mus=20.0, n_groups=groups, t_s=0.5, sigma_t=0.3)
    tgt = workload_custom(22, 20, 8, 40, 0.04, L=21 / 66, mus=20.0, n_groups=groups, t_s=0.5, sigma_t=0.3,
                          seed=5)
    meas = [Solver(tgt, fc_parts=parts).forward(g, 40, tgt.detectors)["curves"] * 0.8 for g in tgt.groups]
    return wl, meas


@pytest.mark.parametrize("parts", [(1, 1), (2, 2)])
def test_discrete_adjoint_is_the_transpose_of_the_tangent_linear_march(parts):
    wl, meas = _case(parts)
    S = Solver(wl, fc_parts=parts)
    rng = np.random.default_rng(11)
    da = rng.standard_normal((wl.grid.ny, wl.grid.nx))
    db = rng.standard_normal((wl.grid.ny, wl.grid.nx))
    for k, g in enumerate(wl.groups):
        _, ga, gb = S.discrete_adjoint_gradient(g, wl.n_steps, wl.detectors, meas[k])
        dJa = S.tangent_linear_objective(g, wl.n_steps, wl.detectors, meas[k], da, 0 * db)
        dJb = S.tangent_linear_objective(g, wl.n_steps, wl.detectors, meas[k], 0 * da, db)
        ea = abs(float((ga * da).sum()) - dJa) / abs(dJa)
        eb = abs(float((gb * db).sum()) - dJb) / abs(dJb)
        print(f"parts {parts} group {k}: dot-product identity a {ea:.1e}, b {eb:.1e}")
        assert ea < 1e-8 and eb < 1e-8


def test_discrete_adjoint_matches_central_differences():
    wl, meas = _case(groups=1)
    S = Solver(wl)
    J, ga, gb = S.discrete_adjoint_gradient(wl.groups[0], wl.n_steps, wl.detectors, meas[0])
    rng = np.random.default_rng(3)
    da = rng.standard_normal(ga.shape)

    def J_of(mua):
        Sp = Solver(dataclasses.replace(wl, mua=mua))
        return Sp.objective(Sp.forward(wl.groups[0], wl.n_steps, wl.detectors)["curves"], meas[0])

    # J is nearly linear in a over this range, while the rounding of the
    # FFT-based march adds noise of ~1e-11 relative to J, which central
    # differences divide by eps: their error falls from 2e-3 at eps = 1e-6
    # to 1.6e-7 at eps = 1e-2, so the large step is the accurate one.
    eps = 1e-2
    fd = (J_of(wl.mua + eps * da) - J_of(wl.mua - eps * da)) / (2 * eps)
    rel = abs(fd - float((ga * da).sum())) / abs(fd)
    print(f"discrete adjoint vs central differences: {rel:.1e}")
    assert rel < 1e-5
    # a single node, well inside: the exact nodal derivative
    j, i = wl.grid.ny // 2, wl.grid.nx // 2
    e = np.zeros_like(ga)
    e[j, i] = 1.0
    fd1 = (J_of(wl.mua + 1e-2 * e) - J_of(wl.mua - 1e-2 * e)) / 2e-2
    assert abs(fd1 - ga[j, i]) < 1e-5 * abs(ga).max()
