"""Pins of the oracle's centred Green's function, Poisson kernel and radial sampler.

Independent references: the paper's printed G (Supplemental 1.1) evaluated here
with scipy.special, integrated with scipy.integrate.quad; the Poisson-kernel
identity stated with it; the sigma -> 0 limits (Sec. 2.3); a KS test of the
sampled radii.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats


def paper_G(dim, R, sb, r):
    """Supplemental 1.1, G^sigma on the centred ball, from scipy's Bessel functions."""
    s = math.sqrt(sb)
    if dim == 2:
        if sb == 0.0:
            return math.log(R / r) / (2 * math.pi)
        # K0(rs) - K0(Rs)/I0(Rs) I0(rs), with exponentially scaled Bessels
        q = special.k0(r * s) - special.k0e(R * s) / special.i0e(R * s) * special.i0e(r * s) * \
            math.exp(r * s - 2 * R * s)
        return q / (2 * math.pi)
    if sb == 0.0:
        return (1 / r - 1 / R) / (4 * math.pi)
    q = math.exp(-r * s) / r - math.exp(-R * s) / R * (math.sinh(r * s) / (r * s)) * \
        ((R * s) / math.sinh(R * s))
    return q / (4 * math.pi)


def sphere_area(dim, r):
    return 2 * math.pi * r if dim == 2 else 4 * math.pi * r * r


def radial_density(dim, R, sb, r):
    return sphere_area(dim, r) * paper_G(dim, R, sb, r)


CASES = [(d, R, sb) for d in (2, 3) for R in (0.01, 0.3, 1.0) for sb in (1e-6, 0.5, 10.0, 60.0, 900.0)]


def _quad(fn, a, b, peak=None):
    pts = [p for p in (peak,) if p is not None and a < p < b]
    v, _ = integrate.quad(fn, a, b, points=pts or None, limit=400, epsabs=0, epsrel=1e-12)
    return v


@pytest.mark.parametrize("dim,R,sb", CASES)
def test_G_matches_printed_form(orc, dim, R, sb):
    for rho in (1e-3, 0.1, 0.5, 0.9, 0.999):
        r = rho * R
        want = paper_G(dim, R, sb, r)
        got = orc.green_G(dim, R, sb, r)
        assert got == pytest.approx(want, rel=1e-9, abs=1e-300)


@pytest.mark.parametrize("dim,R,sb", CASES)
def test_norm_is_integral_of_G(orc, dim, R, sb):
    peak = min(R / 2, 1.0 / math.sqrt(sb))
    want = _quad(lambda r: radial_density(dim, R, sb, r), 0.0, R, peak)
    assert orc.green_norm(dim, R, sb) == pytest.approx(want, rel=1e-9)


@pytest.mark.parametrize("dim,R,sb", CASES)
def test_poisson_kernel_identity(orc, dim, R, sb):
    # Supplemental 1.1: P = (1 - sigma |G|) / |dB|
    P = orc.green_poisson(dim, R, sb)
    G = orc.green_norm(dim, R, sb)
    assert P * sphere_area(dim, R) == pytest.approx(1.0 - sb * G, rel=1e-10, abs=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_laplace_limits(orc, dim):
    # sigma -> 0: |G| = R^2 / (2n), P = 1/|dB| (Sec. 2.3)
    R = 0.7
    assert orc.green_norm(dim, R, 1e-14) == pytest.approx(R * R / (2 * dim), rel=1e-10)
    assert orc.green_poisson(dim, R, 0.0) == pytest.approx(1 / sphere_area(dim, R), rel=1e-14)
    # radial CDF at sigma -> 0: 3D 3 rho^2 - 2 rho^3, 2D rho^2 (1 - 2 ln rho)
    for rho in (0.01, 0.2, 0.5, 0.8, 0.99):
        got = orc.green_cdf(dim, R, 1e-14, rho * R)
        want = 3 * rho ** 2 - 2 * rho ** 3 if dim == 3 else rho ** 2 * (1 - 2 * math.log(rho))
        assert got == pytest.approx(want, rel=1e-9)


A_VALUES = [1e-4, 0.3, 0.99, 1.01, 1.99, 2.01, 3.0, 8.0, 40.0, 250.0]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("a", A_VALUES)
def test_cdf_is_normalised_integral(orc, dim, a):
    R = 0.5
    sb = (a / R) ** 2
    peak = min(0.5 * R, R / a)
    total = _quad(lambda r: radial_density(dim, R, sb, r), 0.0, R, peak)
    for rho in (1e-3, 0.02, 0.1, 0.3, 0.5, 0.7, 0.95):
        r = rho * R
        part = _quad(lambda t: radial_density(dim, R, sb, t), 0.0, r, peak if peak < r else None)
        want = part / total
        got = orc.green_cdf(dim, R, sb, r)
        assert got == pytest.approx(want, rel=1e-8, abs=1e-14)
        # the density is the derivative of the CDF
        assert orc.green_pdf(dim, R, sb, r) == pytest.approx(
            radial_density(dim, R, sb, r) / total, rel=1e-8, abs=1e-12)
    assert orc.green_cdf(dim, R, sb, 0.0) == 0.0
    assert orc.green_cdf(dim, R, sb, R) == 1.0


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("a", [1e-3, 0.5, 1.5, 2.5, 7.0, 60.0])
def test_inverse_cdf_roundtrip(orc, dim, a):
    R = 1.3
    sb = (a / R) ** 2
    for u in (1e-9, 1e-4, 0.01, 0.25, 0.5, 0.75, 0.99, 1 - 1e-7):
        r = orc.green_inv(dim, R, sb, u)
        assert 0.0 < r < R
        assert orc.green_cdf(dim, R, sb, r) == pytest.approx(u, rel=1e-11, abs=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("a", [0.2, 4.0])
def test_sampled_radii_ks(orc, dim, a):
    # radii drawn through F^{-1} follow the printed density (KS against quad CDF)
    R = 1.0
    sb = a * a
    rng = np.random.default_rng(5)
    u = rng.uniform(size=1500)
    r = np.array([orc.green_inv(dim, R, sb, x) for x in u])
    total = _quad(lambda t: radial_density(dim, R, sb, t), 0.0, R, min(0.5, 1 / a))

    def cdf(x):
        return np.array([_quad(lambda t: radial_density(dim, R, sb, t), 0.0, xi) / total
                         for xi in np.atleast_1d(x)])

    res = stats.kstest(r, cdf)
    assert res.pvalue > 1e-3
