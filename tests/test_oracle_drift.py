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


def _p1_moment(dim, R, sb, k):
    """E[r^k] under y ~ G/|G| on the centred ball, by scipy quadrature of the printed G."""
    from scipy import integrate, special
    s = math.sqrt(sb)
    if dim == 3:
        def G(r):
            return math.sinh(s * (R - r)) / (4 * math.pi * r * math.sinh(s * R)) if sb > 0 else \
                (1 / r - 1 / R) / (4 * math.pi)
        w = lambda r: 4 * math.pi * r * r * G(r)
    else:
        def G(r):
            return (special.k0(s * r) - special.k0(s * R) / special.i0(s * R) * special.i0(s * r)) / (2 * math.pi)
        w = lambda r: 2 * math.pi * r * G(r)
    num = integrate.quad(lambda r: r ** k * w(r), 0, R, limit=200)[0]
    den = integrate.quad(w, 0, R, limit=200)[0]
    return num / den


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("lam", [0.97, 0.5])
@pytest.mark.parametrize("R,sb", [(0.3, 1.0), (0.1, 1000.0), (0.5, 50.0)])
def test_mixture_sample_keeps_expectations(orc, dim, lam, R, sb):
    """Reading R22: over the radius uniform u, E[mixw] = 1 and E[mixw r^k] = E_{G/|G|}[r^k]
    (the density ratio undoes the mixture), by midpoint quadrature in u against scipy
    quadrature of the printed G."""
    n = 40000
    u = (np.arange(n) + 0.5) / n
    rw = np.array([orc.mix_radius(dim, R, sb, x, lam) for x in u])
    r, w = rw[:, 0], rw[:, 1]
    assert w.mean() == pytest.approx(1.0, abs=2e-5)
    for k in (1, 2):
        assert (w * r ** k).mean() == pytest.approx(_p1_moment(dim, R, sb, k), rel=1e-4)
    # the part u >= lam is a uniform radius
    j = np.searchsorted(u, lam)
    assert np.allclose(r[j:], R * (u[j:] - lam) / (1 - lam), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_mixture_bounds_the_log_derivative_factor(orc, dim):
    """Reading R22: mixw |G'/G| R stays bounded over the whole radius range (both ends
    included), while |G'/G| R under the plain sample G/|G| is unbounded (it grows without
    limit as u -> 0 and u -> 1)."""
    R, sb = 0.4, 30.0
    u = np.concatenate([np.logspace(-12, -2, 60), np.linspace(0.01, 0.99, 99), 1 - np.logspace(-2, -12, 60)])
    for lam in (0.97, 0.5):
        worst = max(orc.mix_radius(dim, R, sb, x, lam)[1] * orc.green_dlog(dim, R, sb,
                                                                           orc.mix_radius(dim, R, sb, x, lam)[0]) * R
                    for x in u)
        assert worst < 60.0 / (1.0 - lam), (lam, worst)
    plain = max(orc.green_dlog(dim, R, sb, orc.green_inv(dim, R, sb, x)) * R for x in u)
    assert plain > 1e4


def test_per_ball_bound_keeps_the_mean(orc):
    """Reading R23: the drift bound B only changes each ball's delta-tracking bound
    (max(sigma_bar, 10 B / R)); the estimate's expectation does not move (B = 0, the exact
    bound 1.5, and 6)."""
    base = W.cube3d_literal_problem()
    pts = W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 16, 8)]
    sb = orc.sigma_bar(base, 64)[0]
    res = []
    for j, B in enumerate((0.0, 1.5, 6.0)):
        p = dict(base)
        p["drift_bound"] = B
        acc, _ = orc.solve(p, pts, 2048, seed=30 + j, eps=1e-4, sigma_bar=sb)
        res.append(orc.finalize(acc))
    for k in (1, 2):
        ok, nout, mz = four_se_rule(combined_z(res[0][0], res[0][2], res[k][0], res[k][2]))
        assert ok, (k, nout, mz)


def _spread_ratio(u):
    """Per point: sample standard deviation of one walk's estimate over all walks divided by
    the one over the first 1024 (SE * sqrt(N) at N = 2^14 against N = 2^10)."""
    return np.array([np.std(x) / np.std(x[:1024]) for x in u])


@pytest.mark.parametrize("which", ["plain", "extra_drift", "gradient"])
def test_walk_spread_is_constant_in_n(orc, which):
    """SE * sqrt(N) constant over N = 2^10 .. 2^14 (a finite variance): the plain walk on the
    3D workload, the extra-drift walk on its literal drift (readings R22, R23), and the
    gradient walk's components (reading R22 on the first ball)."""
    n = 1 << 14
    if which == "gradient":
        prob = W.cube3d_problem()
        pts = W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 8, 51)]
        _, g, _ = orc.walks_grad(prob, pts, n, seed=52, eps=1e-4, sigma_bar=orc.sigma_bar(prob, 64)[0])
        r = _spread_ratio(g.reshape(-1, n))
        assert 0.85 < np.median(r) < 1.15, r
        return
    prob = W.cube3d_problem() if which == "plain" else W.cube3d_literal_problem()
    pts = W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 12, 53)]
    u, _ = orc.walks(prob, pts, n, seed=54, eps=1e-4, sigma_bar=orc.sigma_bar(prob, 64)[0])
    r = _spread_ratio(u)
    assert 0.85 < np.median(r) < 1.15 and r.max() < 1.5, r
