"""Pins of the oracle's spatial-gradient estimator (Supplemental Sec. 2 and 1.3).

The printed centre gradients of G and P are checked against finite differences
of the ball's Green's function and Poisson kernel for an off-centre x, written
independently as their eigenfunction series (spherical harmonics with modified
spherical Bessel functions in 3D, Fourier modes with I_m, K_m in 2D, from
scipy.special) and, for sigma_bar = 0, as the textbook image-charge closed
forms.  The series at the centre must reproduce the oracle's centred G and the
delta-tracking P, which pins their normalisation.  The whole estimator is then
pinned by its mean against exact gradients of solutions with closed forms.
"""
import math

import numpy as np
import pytest
from scipy import special as sp

import workloads as W
from tests.stats_util import combined_z, four_se_rule


def _g_series(dim, R, sb, xlen, cosang, r):
    """G(x, y) of Lap - sb on the ball |.| < R, |x| = xlen, |y| = r, angle cos = cosang."""
    k = math.sqrt(sb)
    lo, hi = min(xlen, r), max(xlen, r)
    tot = 0.0
    if dim == 3:
        for l in range(40):
            il_lo = sp.spherical_in(l, k * lo)
            term = il_lo * (sp.spherical_kn(l, k * hi) -
                            sp.spherical_kn(l, k * R) * sp.spherical_in(l, k * hi) / sp.spherical_in(l, k * R))
            tot += (2 * l + 1) * term * sp.eval_legendre(l, cosang)
        return k * tot / (2.0 * math.pi ** 2)
    th = math.acos(max(-1.0, min(1.0, cosang)))
    for m in range(40):
        term = sp.iv(m, k * lo) * (sp.kv(m, k * hi) - sp.kv(m, k * R) * sp.iv(m, k * hi) / sp.iv(m, k * R))
        tot += (1.0 if m == 0 else 2.0) * term * math.cos(m * th)
    return tot / (2.0 * math.pi)


def _p_series(dim, R, sb, xlen, cosang):
    k = math.sqrt(sb)
    tot = 0.0
    if dim == 3:
        for l in range(40):
            tot += (2 * l + 1) * sp.spherical_in(l, k * xlen) / sp.spherical_in(l, k * R) * sp.eval_legendre(l, cosang)
        return tot / (4.0 * math.pi * R * R)
    th = math.acos(max(-1.0, min(1.0, cosang)))
    for m in range(40):
        tot += (1.0 if m == 0 else 2.0) * sp.iv(m, k * xlen) / sp.iv(m, k * R) * math.cos(m * th)
    return tot / (2.0 * math.pi * R)


def _g_harmonic(dim, R, x, y):
    """Dirichlet Green's function of the Laplacian on the ball (image point y* = R^2 y/|y|^2)."""
    ny = np.linalg.norm(y)
    ys = R * R * y / ny ** 2
    if dim == 3:
        return (1.0 / np.linalg.norm(x - y) - R / (ny * np.linalg.norm(x - ys))) / (4 * math.pi)
    return (-math.log(np.linalg.norm(x - y)) + math.log(ny * np.linalg.norm(x - ys) / R)) / (2 * math.pi)


def _p_harmonic(dim, R, x, z):
    if dim == 3:
        return (R * R - x @ x) / (4 * math.pi * R * np.linalg.norm(x - z) ** 3)
    return (R * R - x @ x) / (2 * math.pi * R * np.linalg.norm(x - z) ** 2)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("R,sb", [(0.3, 4.0), (0.5, 60.0), (0.05, 900.0), (1.0, 2.5e-3)])
def test_centre_gradients_match_series_differences(orc, dim, R, sb):
    h = 1e-5 * R
    for rho in (0.05, 0.3, 0.6, 0.9):
        r = rho * R
        g0 = orc.green_G(dim, R, sb, r)
        # the series at the centre is the centred G (normalisation pin)
        assert abs(_g_series(dim, R, sb, 0.0, 1.0, r) - g0) <= 1e-10 * abs(g0)
        # derivative along (y - x)/r: x = +-h along y's direction
        dg = (_g_series(dim, R, sb, h, 1.0, r) - _g_series(dim, R, sb, h, -1.0, r)) / (2 * h)
        gG, gP = orc.green_grad_ratios(dim, R, sb, r)
        assert abs(gG * g0 - dg) <= 2e-6 * abs(dg), (rho, gG * g0, dg)
    # the Poisson kernel: centred value is P^dB / |dB| with P^dB = 1 - sb |G|
    area = 2 * math.pi * R if dim == 2 else 4 * math.pi * R * R
    p0 = (1.0 - sb * orc.green_norm(dim, R, sb)) / area
    assert abs(_p_series(dim, R, sb, 0.0, 1.0) - p0) <= 1e-10 * p0
    dp = (_p_series(dim, R, sb, h, 1.0) - _p_series(dim, R, sb, h, -1.0)) / (2 * h)
    gG, gP = orc.green_grad_ratios(dim, R, sb, 0.5 * R)
    assert abs(gP * p0 - dp) <= 2e-6 * abs(dp)


@pytest.mark.parametrize("dim", [2, 3])
def test_centre_gradients_laplace_limit(orc, dim):
    R, h = 0.7, 1e-6
    e = np.zeros(dim)
    e[0] = 1.0
    for rho in (0.1, 0.5, 0.85):
        y = rho * R * e
        g0 = _g_harmonic(dim, R, np.zeros(dim), y)
        dg = (_g_harmonic(dim, R, h * e, y) - _g_harmonic(dim, R, -h * e, y)) / (2 * h)
        gG, gP = orc.green_grad_ratios(dim, R, 0.0, rho * R)
        assert abs(gG * g0 - dg) <= 1e-6 * abs(dg)
        assert abs(orc.green_G(dim, R, 0.0, rho * R) - g0) <= 1e-12 * abs(g0)
    z = R * e
    p0 = _p_harmonic(dim, R, np.zeros(dim), z)
    dp = (_p_harmonic(dim, R, h * e, z) - _p_harmonic(dim, R, -h * e, z)) / (2 * h)
    gG, gP = orc.green_grad_ratios(dim, R, 0.0, 0.5 * R)
    assert abs(gP * p0 - dp) <= 1e-6 * abs(dp)
    # the screened ratios tend to the Laplace ones as sb -> 0
    for rho in (0.2, 0.7):
        a = orc.green_grad_ratios(dim, R, 1e-8, rho * R)
        b = orc.green_grad_ratios(dim, R, 0.0, rho * R)
        assert np.allclose(a, b, rtol=1e-6)


def test_walk_grad_value_matches_the_plain_walk(orc):
    """The gradient walk is the walk of Alg. 1 except for its first ball, which draws the
    mixture sample of reading R22 (G/|G| weight 1/2) and carries its density ratio: the
    value estimate keeps the plain walk's expectation (4 combined standard errors), walks
    that leave the first ball the same way take the same number of steps on average, and
    every gradient is finite."""
    prob = W.cube3d_problem()
    sb = orc.sigma_bar(prob)[0]
    pts = W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 12, 44)].astype(np.float64)
    u0, k0 = orc.walks(prob, pts, 4096, seed=9, eps=1e-4, sigma_bar=sb)
    u1, g, k1 = orc.walks_grad(prob, pts, 4096, seed=10, eps=1e-4, sigma_bar=sb)
    m0, s0 = u0.mean(1), u0.std(1, ddof=1) / 64.0
    m1, s1 = u1.mean(1), u1.std(1, ddof=1) / 64.0
    ok, nout, mz = four_se_rule(combined_z(m0, s0, m1, s1))
    assert ok, (nout, mz)
    assert abs(k1.mean() / k0.mean() - 1.0) < 0.02
    assert np.all(np.isfinite(g))


def test_walk_grad_in_shell_is_undefined(orc):
    prob = W.square2d_problem()
    sb = orc.sigma_bar(prob)[0]
    u, g, k, _ = orc.walk_grad(prob, np.array([0.5, 1e-4]), 0, 0, 0, 1e-3, sb)
    assert k == 0 and np.all(np.isnan(g))


GRAD_CASES = {
    "laplace_disk": (W.laplace_disk_problem, lambda p: W.laplace_disk_exact_grad(*p),
                     lambda: W.uniform_in_ball(2, 8, [0, 0], 1.0, seed=3, margin=0.2), 3000, 1e-4),
    "laplace_ball": (W.laplace_ball_problem, lambda p: W.laplace_ball_exact_grad(*p),
                     lambda: W.uniform_in_ball(3, 6, [0, 0, 0], 1.0, seed=4, margin=0.2), 3000, 1e-4),
    "screened_ball": (W.screened_ball_problem, lambda p: W.screened_ball_exact_grad(9.0, *p),
                      lambda: W.uniform_in_ball(3, 6, [0, 0, 0], 1.0, seed=5, margin=0.2), 3000, 1e-4),
    "square2d": (W.square2d_problem, lambda p: W.square2d_exact_grad(*p),
                 lambda: W.cell_centres(2, 32)[:, W.seeded_subset(1024, 8, 5)], 4000, 1e-4),
    "cube3d": (W.cube3d_problem, lambda p: W.cube3d_exact_grad(*p),
               lambda: W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 6, 6)], 3000, 1e-4),
    "hifreq": (W.hifreq_alpha_problem, lambda p: W.hifreq_alpha_exact_grad(*p),
               lambda: W.cell_centres(2, 16)[:, W.seeded_subset(256, 6, 8)], 3000, 1e-4),
}


@pytest.mark.parametrize("name", list(GRAD_CASES))
def test_gradient_estimator_matches_exact_gradient(orc, name):
    """E[grad estimate] = grad u (Supplemental Sec. 2) on solutions with closed forms; cube3d and
    hifreq carry the -u grad gamma term (alpha and Phi vary)."""
    mk, exact, ptsf, walks, eps = GRAD_CASES[name]
    prob = mk()
    pts = ptsf()
    sb = orc.sigma_bar(prob)[0]
    m, se, g, gse = orc.solve_grad(prob, pts, walks, seed=1, eps=eps, sigma_bar=sb)
    want = exact(pts.astype(np.float64)).T  # [npts, dim]
    z = ((g - want) / gse).ravel()
    ok, nout, mz = four_se_rule(z)
    assert ok, (name, z)
