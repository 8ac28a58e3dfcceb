"""Pins of the oracle's extra-drift walk (a drift that is not alpha times a gradient).

Not in the paper, which removes only drifts with omega/alpha = grad(Phi) (App. A).
With b = omega_extra/alpha the transformed equation keeps b . grad U; on each ball
it is moved onto the Green's function by parts (G vanishes on the sphere):
    int_B G b . grad U dy = -int_B U (grad_y G . b + G div b) dy,
so a null event at y = x + r dir_y carries the weight
    1 - (sigma' + b . grad gamma + div b)/sigma_bar + |G'(r)/G(r)| (dir_y . b(y))/sigma_bar.
Pinned here: |G'/G| against differences of the centred G; the walk's mean against
closed-form solutions with non-conservative drifts (the cube workload's literal
omega = (sin 2 pi y, cos 2 pi z, 0.5), a 2D rotational drift); invariance in
sigma_bar.
"""
import math

import numpy as np
import pytest

import workloads as W
from tests.stats_util import combined_z, four_se_rule


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("R,sb", [(0.4, 2.0), (0.2, 300.0), (1.0, 1e-3), (0.5, 0.0)])
def test_green_log_derivative(orc, dim, R, sb):
    for rho in (0.05, 0.3, 0.7, 0.95):
        r = rho * R
        h = 1e-6 * R
        d = (math.log(orc.green_G(dim, R, sb, r + h)) - math.log(orc.green_G(dim, R, sb, r - h))) / (2 * h)
        assert abs(orc.green_dlog(dim, R, sb, r) + d) <= 1e-6 * abs(d), (rho, orc.green_dlog(dim, R, sb, r), -d)


def _rot2d_problem():
    """u = sin(pi x) cosh(y) on the unit square, alpha = 1 + 0.5 sin 2 pi x cos 2 pi y,
    sigma = 2 + sin(3x + y), omega = (2 x sin(pi y), y cos(pi x)): curl and divergence
    (2 sin(pi y) + cos(pi x)) both non-zero."""
    p = W.square2d_problem()
    om = [W.sst(W.term(2.0, (W.LIN, 1.0, 0.0), (W.SIN, W.PI, 0.0))),
          W.sst(W.term(1.0, (W.COS, W.PI, 0.0), (W.LIN, 1.0, 0.0)))]
    return W.problem(2, p["domain"], p["alpha"], p["sigma"], p["f"], p["g"], um=p["um"], omega=om)


def _expalpha_problem():
    """alpha = e^{2x} (grad gamma = (1, 0)), omega = (3 y, 0) (curl -3): b . grad gamma = 3 y e^{-2x}
    and div b = -6 y e^{-2x} both matter; u = sin(pi x) cosh(y), sigma = 1."""
    u = W.sst(W.term(1.0, (W.SIN, W.PI, 0.0), (W.COSH, 1.0, 0.0)))
    alpha = W.sst(W.term(1.0, (W.EXP, 2.0, 0.0)))
    om = [W.sst(W.term(3.0, None, (W.LIN, 1.0, 0.0))), W.zero()]
    return W.problem(2, W.box([0, 0], [1, 1]), alpha, W.const(1.0), W.manufactured(), u, um=u, omega=om)


CASES = {
    "square_exp_alpha": (_expalpha_problem, lambda p: W.square2d_exact(*p),
                         lambda: W.cell_centres(2, 32)[:, W.seeded_subset(1024, 32, 4)], 5000),
    "cube3d_literal": (W.cube3d_literal_problem, lambda p: W.cube3d_exact(*p),
                       lambda: W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 12, 6)], 3000),
    "square_rotational": (_rot2d_problem, lambda p: W.square2d_exact(*p),
                          lambda: W.cell_centres(2, 32)[:, W.seeded_subset(1024, 12, 5)], 3000),
}


@pytest.mark.parametrize("name", list(CASES))
def test_extra_drift_walk_matches_exact_solution(orc, name):
    mk, exact, ptsf, walks = CASES[name]
    prob = mk()
    pts = ptsf()
    sb = orc.sigma_bar(prob)[0]
    acc, st = orc.solve(prob, pts, walks, seed=2, eps=1e-4, sigma_bar=sb)
    m, v, se = orc.finalize(acc)
    ok, nout, mz = four_se_rule((m - exact(pts.astype(np.float64))) / se)
    assert ok, (name, (m - exact(pts.astype(np.float64))) / se)
    assert st["capped"] == 0 and st["nonfinite"] == 0


def test_extra_drift_sigma_bar_invariance(orc):
    prob = W.cube3d_literal_problem()
    pts = W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 10, 8)]
    sb = orc.sigma_bar(prob)[0]
    a, _ = orc.solve(prob, pts, 3000, seed=3, eps=1e-4, sigma_bar=sb)
    b, _ = orc.solve(prob, pts, 3000, seed=4, eps=1e-4, sigma_bar=4 * sb)
    m1, _, se1 = orc.finalize(a)
    m2, _, se2 = orc.finalize(b)
    ok, nout, mz = four_se_rule(combined_z(m1, se1, m2, se2))
    assert ok
