"""Pins of the oracle's next-flight walk (Sec. 5.2, Supplemental Algorithm 2) and of
the approximate off-centred Green's function and Poisson kernel it uses
(Supplemental 1.2).

The series of Supplemental 1.2 (the exact kernels; orc_series_G / _P) are pinned
below against their centred forms, the printed single series summed with scipy, the
Laplacian's image kernels, the normal-derivative relation, the screened equation,
and the boundary-value-1 solution that P integrates to.

What the paper fixes about the approximations, checked here:
* they equal the centred G and P of Supplemental 1.1 when x is the ball centre;
* P is the (negative) normal derivative of G on the sphere, as printed;
* for the Laplacian along the ray through the centre (u parallel to v) they equal
  the exact image-charge Green's function and Poisson kernel;
* away from the centre they deviate from the exact kernels (the eigenfunction
  series of Supplemental 1.2, summed with scipy), increasingly with |u|.
The walk itself is pinned where its estimate is exact whatever the off-centre
error: with sigma_bar = sigma' every null weight sigma_bar - sigma' is zero, so
every ball uses only the centred kernels (screened ball; screened square with a
source), and for a Laplace problem the off-centre terms carry a factor
sigma_bar R^2 ~ 1e-5.
"""
import math

import numpy as np
import pytest

import workloads as W
from tests.stats_util import four_se_rule
from tests.test_oracle_grad import _g_harmonic, _g_series, _p_harmonic, _p_series


def _vec(dim, r, ang):
    v = np.zeros(dim)
    v[0], v[1] = r * math.cos(ang), r * math.sin(ang)
    return v


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("R,sb", [(0.5, 60.0), (0.2, 4.0), (1.0, 1e-3)])
def test_offcentre_exact_at_centre(orc, dim, R, sb):
    area = 2 * math.pi * R if dim == 2 else 4 * math.pi * R * R
    u = np.zeros(dim)
    for rho in (0.05, 0.4, 0.9):
        v = _vec(dim, rho * R, 0.7)
        g = orc.offcentre_G(dim, R, sb, u, v)
        assert abs(g - orc.green_G(dim, R, sb, rho * R)) <= 1e-12 * abs(g)
    z = _vec(dim, R, 2.1)
    p = orc.offcentre_P(dim, R, sb, u, z)
    assert abs(p - (1.0 - sb * orc.green_norm(dim, R, sb)) / area) <= 1e-12 * p


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("sb", [60.0, 1e-3])
def test_offcentre_P_is_normal_derivative_of_G(orc, dim, sb):
    """P(x, z) = -dG(x, y)/dn at y = z on the sphere, for the printed forms of both."""
    R, h = 0.5, 1e-6
    for fu, ang in ((0.2, 0.4), (0.5, 1.9), (0.7, 3.0)):
        u = _vec(dim, fu * R, 0.3)
        z = _vec(dim, R, ang)
        n = z / R
        dg = (orc.offcentre_G(dim, R, sb, u, z + h * n) - orc.offcentre_G(dim, R, sb, u, z - h * n)) / (2 * h)
        p = orc.offcentre_P(dim, R, sb, u, z)
        assert abs(p + dg) <= 1e-6 * abs(p), (fu, ang, p, -dg)


@pytest.mark.parametrize("dim", [2, 3])
def test_offcentre_laplace_on_the_radial_line(orc, dim):
    R = 0.8
    for fu, fv in ((0.3, 0.6), (0.7, 0.2), (-0.5, 0.9)):
        u = _vec(dim, fu * R, 0.0)
        v = _vec(dim, fv * R, 0.0)
        g = orc.offcentre_G(dim, R, 0.0, u, v)
        assert abs(g - _g_harmonic(dim, R, u, v)) <= 1e-12 * abs(g)
        z = _vec(dim, R, 0.0 if fu > 0 else math.pi)
        p = orc.offcentre_P(dim, R, 0.0, u, z)
        assert abs(p - _p_harmonic(dim, R, u, z)) <= 1e-12 * abs(p)


@pytest.mark.parametrize("dim", [2, 3])
def test_offcentre_approximation_error_grows_from_the_centre(orc, dim):
    """The approximations against the exact series: close near the centre, far off near the
    sphere (a characterisation of Supplemental 1.2's approximation, not a bound the paper states)."""
    R, sb = 0.5, 4.0

    def worst(fu):
        e = 0.0
        u = _vec(dim, fu * R, 0.0)
        for ang in (0.3, 1.2, 2.5):
            for fr in (0.3, 0.8):
                v = _vec(dim, fr * R, ang)
                c = math.cos(ang)
                gs = _g_series(dim, R, sb, fu * R, c, fr * R)
                e = max(e, abs(orc.offcentre_G(dim, R, sb, u, v) - gs) / abs(gs))
            z = _vec(dim, R, ang)
            ps = _p_series(dim, R, sb, fu * R, math.cos(ang))
            e = max(e, abs(orc.offcentre_P(dim, R, sb, u, z) - ps) / abs(ps))
        return e
    e1, e3, e6 = worst(0.1), worst(0.3), worst(0.6)
    assert e1 < 0.05 and e1 < e3 < e6 and e6 > 0.3, (e1, e3, e6)


# ---------------------------------------------------------------------------
# The series of Supplemental 1.2 (orc_series_G / orc_series_P)
# ---------------------------------------------------------------------------
def _centred_G(dim, R, sb, r):
    """Closed-form centred G (Supplemental 1.1): 3D sinh(k(R-r))/(4 pi r sinh(kR)),
    2D (K0(kr) - K0(kR) I0(kr)/I0(kR)) / (2 pi)."""
    k = math.sqrt(sb)
    if dim == 3:
        return math.sinh(k * (R - r)) / (4 * math.pi * r * math.sinh(k * R))
    from scipy import special as sp
    return (sp.k0(k * r) - sp.k0(k * R) * sp.i0(k * r) / sp.i0(k * R)) / (2 * math.pi)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("R,sb", [(0.5, 60.0), (0.2, 4.0), (1.0, 1e-3), (0.3, 2500.0)])
def test_series_at_centre_are_the_centred_kernels(orc, dim, R, sb):
    """x = c: only the n = 0 term survives and the series are Supplemental 1.1's forms
    (written out here: the screened kernels of the ball about its centre)."""
    k = math.sqrt(sb)
    area = 2 * math.pi * R if dim == 2 else 4 * math.pi * R * R
    u = np.zeros(dim)
    for rho in (0.05, 0.4, 0.9):
        v = _vec(dim, rho * R, 0.7)
        g = orc.series_G(dim, R, sb, u, v)
        assert abs(g - _centred_G(dim, R, sb, rho * R)) <= 1e-10 * abs(g), (rho, g)
    from scipy import special as sp
    p_ref = (k * R / math.sinh(k * R) if dim == 3 else 1.0 / sp.i0(k * R)) / area
    for n in (0, 1, 5):
        p = orc.series_P(dim, R, sb, u, _vec(dim, R, 2.1), n)
        assert abs(p - p_ref) <= 1e-12 * p_ref


def _printed_series_G(dim, R, sb, xlen, cosang, r, nmax=100):
    """The printed single series of Supplemental 1.2 for G, summed with scipy to nmax terms."""
    from scipy import special as sp
    k = math.sqrt(sb)
    lo, hi = min(xlen, r), max(xlen, r)
    tot = 0.0
    for n in range(nmax):
        if dim == 3:
            kn = lambda z: math.sqrt(2.0 / (math.pi * z)) * sp.kv(n + 0.5, z)  # k_0(z) = e^{-z}/z
            t = (2 * n + 1) * sp.eval_legendre(n, cosang) * sp.spherical_in(n, k * lo) * (
                kn(k * hi) - kn(k * R) * sp.spherical_in(n, k * hi) / sp.spherical_in(n, k * R))
        else:
            t = (1.0 if n == 0 else 2.0) * math.cos(n * math.acos(cosang)) * sp.iv(n, k * lo) * (
                sp.kv(n, k * hi) - sp.kv(n, k * R) * sp.iv(n, k * hi) / sp.iv(n, k * R))
        assert math.isfinite(t)
        tot += t
    return tot * (k / (4 * math.pi) if dim == 3 else 1.0 / (2 * math.pi))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("R,sb", [(0.5, 60.0), (0.3, 4.0), (1.0, 20.0)])
def test_series_match_the_printed_single_series(orc, dim, R, sb):
    """Off the centre: the printed series (I(r<) (K(r>) - K(R) I(r>)/I(R)), summed with
    scipy's Bessel functions) equals the oracle's closed-form free-space kernel minus
    the series of the regular part, and the printed P series equals the oracle's."""
    for fu, fv, ang in ((0.2, 0.5, 0.4), (0.45, 0.3, 2.0), (0.5, 0.7, 1.1), (0.1, 0.6, 3.0)):
        u = _vec(dim, fu * R, 0.3)
        v = _vec(dim, fv * R, 0.3 + ang)
        ref = _printed_series_G(dim, R, sb, fu * R, math.cos(ang), fv * R)
        g = orc.series_G(dim, R, sb, u, v)
        assert abs(g - ref) <= 1e-9 * abs(ref), (fu, fv, ang, g, ref)
        z = _vec(dim, R, 0.3 + ang)
        pref = _p_series(dim, R, sb, fu * R, math.cos(ang))
        p = orc.series_P(dim, R, sb, u, z)
        assert abs(p - pref) <= 1e-10 * abs(pref), (fu, ang, p, pref)


@pytest.mark.parametrize("dim", [2, 3])
def test_series_laplace_limit_is_the_image_kernel(orc, dim):
    """sigma_bar = 0, and sigma_bar -> 0: the Laplacian's image-point kernels (closed forms)."""
    R = 0.8
    for sb, tol in ((0.0, 1e-12), (1e-9, 1e-6)):
        for fu, fv, ang in ((0.3, 0.6, 0.5), (0.7, 0.2, 2.2), (0.5, 0.5, 1.0)):
            u = _vec(dim, fu * R, 0.1)
            v = _vec(dim, fv * R, 0.1 + ang)
            g = orc.series_G(dim, R, sb, u, v)
            ref = _g_harmonic(dim, R, u, v)
            assert abs(g - ref) <= tol * abs(ref), (sb, fu, fv, g, ref)
            z = _vec(dim, R, 0.1 + ang)
            p = orc.series_P(dim, R, sb, u, z)
            pref = _p_harmonic(dim, R, u, z)
            assert abs(p - pref) <= tol * abs(pref), (sb, fu, p, pref)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("sb", [60.0, 3.0])
def test_series_P_is_normal_derivative_of_G(orc, dim, sb):
    """The series P (simplified by the Wronskians) is -dG/dn of the series G at the sphere,
    and G vanishes there."""
    R, h = 0.5, 1e-6
    for fu, ang in ((0.2, 0.4), (0.5, 1.9), (0.7, 3.0)):
        u = _vec(dim, fu * R, 0.3)
        z = _vec(dim, R, ang)
        n = z / R
        assert abs(orc.series_G(dim, R, sb, u, z)) <= 1e-12 * abs(orc.series_G(dim, R, sb, u, 0.5 * z))
        dg = (orc.series_G(dim, R, sb, u, z + h * n) - orc.series_G(dim, R, sb, u, z - h * n)) / (2 * h)
        p = orc.series_P(dim, R, sb, u, z)
        assert abs(p + dg) <= 1e-6 * abs(p), (fu, ang, p, -dg)


@pytest.mark.parametrize("dim", [2, 3])
def test_series_G_solves_the_screened_equation(orc, dim):
    """Lap_y G - sigma_bar G = 0 away from y = x (second differences), G(x, y) = G(y, x)."""
    R, sb, h = 0.6, 25.0, 1e-3
    u = _vec(dim, 0.25, 0.4)
    for y in (_vec(dim, 0.3, 2.0), _vec(dim, 0.45, -1.0)):
        g = orc.series_G(dim, R, sb, u, y)
        lap = 0.0
        for i in range(dim):
            e = np.zeros(dim)
            e[i] = h
            lap += orc.series_G(dim, R, sb, u, y + e) + orc.series_G(dim, R, sb, u, y - e) - 2 * g
        lap /= h * h
        assert abs(lap - sb * g) <= 1e-4 * sb * abs(g), (lap, sb * g)
        assert abs(orc.series_G(dim, R, sb, y, u) - g) <= 1e-12 * abs(g)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("nterms", [1, 4, 16, 0])
def test_series_P_integrates_to_the_boundary_solution(orc, dim, nterms):
    """int_dB P(x, z) dz = the solution with boundary value 1, i_0(k r)/i_0(k R) (3D) or
    I_0(k r)/I_0(k R) (2D), for every truncation: the terms n >= 1 integrate to zero."""
    from scipy import special as sp
    R, sb = 0.7, 9.0
    k = math.sqrt(sb)
    for fu in (0.2, 0.6):
        r = fu * R
        exact = (R * math.sinh(k * r) / (r * math.sinh(k * R))) if dim == 3 else sp.i0(k * r) / sp.i0(k * R)
        u = _vec(dim, r, 0.0)
        if dim == 3:
            # axisymmetric about u: dz = 2 pi R^2 dmu
            xs, ws = np.polynomial.legendre.leggauss(64)
            tot = sum(w * orc.series_P(3, R, sb, u, R * np.array([c, math.sqrt(1 - c * c), 0.0]), nterms)
                      for c, w in zip(xs, ws)) * 2 * math.pi * R * R
        else:
            th = (np.arange(256) + 0.5) * 2 * math.pi / 256
            tot = sum(orc.series_P(2, R, sb, u, _vec(2, R, t), nterms) for t in th) * 2 * math.pi * R / 256
        assert abs(tot - exact) <= 1e-9 * exact, (fu, tot, exact)


@pytest.mark.parametrize("dim", [2, 3])
def test_series_walk_radius_follows_the_free_space_kernel(orc, dim):
    """The series walk's in-ball distance r (reading R24) has density proportional to
    Phi(r) r^{d-1} on [0, r_m] (Phi: e^{-kr}/(4 pi r) in 3D, K_0(kr)/(2 pi) in 2D): its CDF,
    integrated with scipy, equals the uniform it was drawn from; h(t) is that mass."""
    from scipy import integrate
    from scipy import special as sp
    dens = (lambda r, k: r * math.exp(-k * r)) if dim == 3 else (lambda r, k: r * sp.k0(k * r))
    for sb, rm in ((45.0, 0.3), (4.0, 0.8), (900.0, 0.5), (1e-4, 0.2)):
        k = math.sqrt(sb)
        tot = integrate.quad(dens, 0, rm, args=(k,), epsabs=0, epsrel=1e-12, limit=200)[0]
        assert abs(orc.nf_h(dim, k * rm) - k * k * tot) <= 1e-10 * k * k * tot
        for u in (1e-6, 0.1, 0.5, 0.9, 0.999999):
            r = orc.nf_free_radius(dim, sb, rm, u)
            assert 0.0 <= r <= rm
            F = integrate.quad(dens, 0, r, args=(k,), epsabs=0, epsrel=1e-12, limit=200)[0] / tot
            assert abs(F - u) <= 1e-9, (sb, rm, u, F)


NF_CASES = {
    # sigma_bar = sigma' (constant): every inner series stops after its first term
    "screened_ball": (W.screened_ball_problem, lambda p: W.screened_ball_exact(9.0, *p),
                      lambda: W.uniform_in_ball(3, 8, [0, 0, 0], 1.0, seed=4, margin=0.05), 9.0, 3000),
    "screened_square": (W.screened_square_problem, lambda p: W.screened_square_exact(*p),
                        lambda: W.uniform_in_box(2, 8, 0.05, 0.95, seed=3), 4.0, 3000),
    # Laplace with the sigma_bar floor: off-centre terms are O(sigma_bar R^2)
    "laplace_disk": (W.laplace_disk_problem, lambda p: W.laplace_disk_exact(*p),
                     lambda: W.uniform_in_ball(2, 8, [0, 0], 1.0, seed=1, margin=0.05), None, 3000),
    "laplace_ball": (W.laplace_ball_problem, lambda p: W.laplace_ball_exact(*p),
                     lambda: W.uniform_in_ball(3, 8, [0, 0, 0], 1.0, seed=2, margin=0.05), None, 3000),
}


@pytest.mark.parametrize("name", list(NF_CASES))
def test_next_flight_exact_cases(orc, name):
    mk, exact, ptsf, sb, walks = NF_CASES[name]
    prob = mk()
    pts = ptsf()
    if sb is None:
        sb = orc.sigma_bar(prob)[0]
    uh, st, inner = orc.walks_nf(prob, pts, walks, seed=3, eps=1e-4, sigma_bar=sb)
    m = uh.mean(1)
    se = uh.std(1, ddof=1) / math.sqrt(walks)
    ok, nout, mz = four_se_rule((m - exact(pts.astype(np.float64))) / se)
    assert ok, (name, (m - exact(pts.astype(np.float64))) / se)
    assert np.all(st > 0) and np.all(inner >= st)


def test_next_flight_distance_queries_do_not_grow_with_sigma_bar(orc):
    """Sec. 5.2, Fig. 12: raising sigma_bar multiplies the delta-tracking walk's distance
    queries but leaves the next-flight walk's unchanged."""
    prob = W.screened_square_problem()
    pts = W.uniform_in_box(2, 6, 0.2, 0.8, seed=5)
    counts = {}
    for sb in (4.0, 400.0):
        _, st_nf, _ = orc.walks_nf(prob, pts, 400, seed=1, eps=1e-3, sigma_bar=sb)
        _, st_dt = orc.walks(prob, pts, 400, seed=1, eps=1e-3, sigma_bar=sb)
        counts[sb] = (st_nf.mean(), st_dt.mean())
    assert counts[400.0][1] > 2.5 * counts[4.0][1], counts
    assert abs(counts[400.0][0] / counts[4.0][0] - 1.0) < 0.1


def test_next_flight_stream_layout(orc):
    """Walk ids continue streams; the walk at sigma_bar = sigma' uses one inner iteration per ball."""
    prob = W.screened_ball_problem()
    x = np.array([0.1, -0.2, 0.3])
    for j in range(8):
        u, k, m, fl = orc.walk_nf(prob, x, 2, j, 4, 1e-4, 9.0)
        assert fl == 0 and m == k
    a, sa, ia = orc.walks_nf(prob, x[:, None], 6, seed=4, eps=1e-4, sigma_bar=9.0)
    b, sb_, ib = orc.walks_nf(prob, x[:, None], 3, seed=4, eps=1e-4, sigma_bar=9.0, walk_offset=3)
    assert np.array_equal(a[:, 3:], b) and np.array_equal(sa[:, 3:], sb_)


def test_next_flight_in_shell_returns_boundary_value(orc):
    prob = W.square2d_problem()
    sb = orc.sigma_bar(prob)[0]
    u, k, m, fl = orc.walk_nf(prob, np.array([0.5, 1e-4]), 0, 0, 0, 1e-3, sb)
    d, xb = orc.distance(prob, np.array([0.5, 1e-4]))
    assert k == 0 and m == 0 and abs(u - W.square2d_exact(*xb)) <= 1e-12



@pytest.mark.parametrize("name", ["cube3d", "square2d"])
def test_next_flight_with_series_is_unbiased_where_sigma_varies(orc, name):
    """With the series kernels (truncated at 8 terms) and free-space-kernel in-ball points
    the next-flight walk's mean agrees with the exact solution where sigma' varies and the
    null weights do not vanish; truncation keeps the kernels' low harmonics, and the smooth
    boundary data and sources carry almost nothing above them.  (The printed
    approximations are checked only where they are exact.)"""
    if name == "cube3d":
        prob, exact = W.cube3d_problem(), W.cube3d_exact
        pts = W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 12, 2)]
        sb = orc.sigma_bar(prob, 64)[0]
    else:
        prob, exact = W.square2d_problem(), W.square2d_exact
        pts = W.cell_centres(2, 32)[:, W.seeded_subset(1024, 12, 1)]
        sb = orc.sigma_bar(prob)[0]
    walks = 8192
    uh, st, inner = orc.walks_nf(prob, pts, walks, seed=7, eps=1e-4, sigma_bar=sb, series_terms=8)
    m = uh.mean(1)
    se = uh.std(1, ddof=1) / math.sqrt(walks)
    ex = np.array([exact(*pts[:, i]) for i in range(pts.shape[1])])
    ok, nout, mz = four_se_rule((m - ex) / se)
    assert ok, (m - ex) / se
    assert np.all(np.isfinite(uh)) and np.all(inner >= st)
