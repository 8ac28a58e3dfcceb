"""Pins of the oracle's distance and closest-point queries (Alg. 1 DistanceToBoundary).

Reference: brute force over a dense sampling of each boundary.
"""
import math

import numpy as np
import pytest

import workloads as W


def boundary_samples(dom, dim, n=400):
    k = dom["kind"]
    p = dom["p"]
    if dim == 2:
        t = np.linspace(0, 2 * math.pi, 20 * n, endpoint=False)
        circ = np.stack([np.cos(t), np.sin(t)], axis=1)
    else:
        rng = np.random.default_rng(0)
        v = rng.normal(size=(40 * n, 3))
        circ = v / np.linalg.norm(v, axis=1, keepdims=True)
    c = np.array(p[:dim])
    if k == "box":
        lo, hi = np.array(p[:dim]), np.array(p[3:3 + dim])
        s = []
        g = np.linspace(0, 1, 4 * n if dim == 2 else 60)
        for d in range(dim):
            for face in (lo[d], hi[d]):
                if dim == 2:
                    pts = np.zeros((len(g), 2))
                    pts[:, d] = face
                    o = 1 - d
                    pts[:, o] = lo[o] + g * (hi[o] - lo[o])
                else:
                    o = [e for e in range(3) if e != d]
                    A, B = np.meshgrid(g, g)
                    pts = np.zeros((A.size, 3))
                    pts[:, d] = face
                    pts[:, o[0]] = lo[o[0]] + A.ravel() * (hi[o[0]] - lo[o[0]])
                    pts[:, o[1]] = lo[o[1]] + B.ravel() * (hi[o[1]] - lo[o[1]])
                s.append(pts)
        return np.concatenate(s)
    if k == "ball":
        return c + p[3] * circ
    if k == "annulus":
        return np.concatenate([c + p[3] * circ, c + p[4] * circ])
    if k == "rounded_box":
        half = np.array(p[3:3 + dim])
        rc = p[6]
        inner = half - rc
        # Minkowski sum boundary: points at distance rc from the inner box
        q = circ * rc
        g = np.linspace(-1, 1, 2 * n)
        s = []
        for d in range(dim):
            o = 1 - d
            for sgn in (-1, 1):
                pts = np.zeros((len(g), 2))
                pts[:, d] = sgn * half[d]
                pts[:, o] = g * inner[o]
                s.append(c + pts)
        for sx in (-1, 1):
            for sy in (-1, 1):
                corner = np.array([sx * inner[0], sy * inner[1]])
                arc = q[(q[:, 0] * sx >= 0) & (q[:, 1] * sy >= 0)]  # outward quarter arc only
                s.append(c + corner + arc)
        return np.concatenate(s)
    raise ValueError(k)


DOMAINS = [
    (2, W.box([0, 0], [1, 2])),
    (3, W.box([0, 0, 0], [1, 1, 2])),
    (2, W.ball([0.3, -0.2], 1.5)),
    (3, W.ball([0.1, 0.2, 0.3], 0.8)),
    (2, W.annulus([0.5, 0.5], 0.4, 1.1)),
    (2, W.rounded_box([0.2, 0.1], [1.0, 0.6], 0.25)),
]


@pytest.mark.parametrize("dim,dom", DOMAINS)
def test_distance_and_closest_point(orc, dim, dom):
    prob = W.problem(dim, dom, W.const(1), W.zero(), W.zero(), W.zero())
    bs = boundary_samples(dom, dim)
    lo = bs.min(axis=0)
    hi = bs.max(axis=0)
    rng = np.random.default_rng(4)
    tested = 0
    for _ in range(400):
        x = rng.uniform(lo, hi)
        d, xb = orc.distance(prob, x)
        if d <= 0:
            continue
        tested += 1
        brute = np.linalg.norm(bs - x, axis=1).min()
        spacing = 0.02 if dim == 2 else 0.05
        assert d == pytest.approx(brute, abs=spacing)
        assert d <= brute + 1e-12
        # the closest point lies at distance d and on the boundary (its own distance is 0)
        assert np.linalg.norm(xb - x) == pytest.approx(d, rel=1e-12, abs=1e-12)
        d2, _ = orc.distance(prob, xb)
        assert abs(d2) < 1e-12
    assert tested > 50


# ---------------------------------------------------------------------------
# signed-distance CSG domains (Sec. 7.2)
# ---------------------------------------------------------------------------
def _inside_points(orc, prob, n, seed, margin=0.0):
    dim = prob["dim"]
    lo = np.array(prob["domain"]["p"][:dim])
    hi = np.array(prob["domain"]["p"][3:3 + dim])
    X = lo + (hi - lo) * np.random.default_rng(seed).uniform(size=(n, dim))
    d = np.array([orc.distance(prob, x)[0] for x in X])
    return X[d > margin], X, d


@pytest.mark.parametrize("dim", [2, 3])
def test_csg_single_primitive_matches_analytic_domains(orc, dim):
    """A one-node CSG list of a sphere / rounded box is the ball / rounded-box domain."""
    c = [0.1, -0.2, 0.3][:dim]
    cases = [(W.csg([-2] * dim, [2] * dim, ("sphere", "union", c + [0.0] * (3 - dim) + [0.8])), W.ball(c, 0.8)),
             (W.csg([-2] * dim, [2] * dim, ("box", "union", c + [0.0] * (3 - dim) + [0.7, 0.5, 0.4][:dim] +
                                            [0.0] * (3 - dim) + [0.1])),
              W.rounded_box(c, [0.7, 0.5, 0.4][:dim], 0.1))]
    rng = np.random.default_rng(dim)
    for dom_csg, dom_ref in cases:
        pa = W.problem(dim, dom_csg, W.const(1.0), W.zero(), W.zero(), W.zero())
        pb = W.problem(dim, dom_ref, W.const(1.0), W.zero(), W.zero(), W.zero())
        for x in np.array(c) + rng.uniform(-0.6, 0.6, size=(200, dim)):
            da, xa = orc.distance(pa, x)
            db, xb = orc.distance(pb, x)
            if db > 1e-9:
                assert abs(da - db) <= 1e-12 and np.allclose(xa, xb, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_csg_ball_stays_inside(orc, dim):
    """The ball of radius -sdf(x) contains no outside point (min/max of exact primitive
    distances bound the distance from below; the sign is exact)."""
    prob = W.csg_laplace_problem(dim)
    inside, X, d = _inside_points(orc, prob, 60000 if dim == 3 else 30000, seed=1)
    outside = X[d < 0]
    for x in inside[:300]:
        R = orc.distance(prob, x)[0]
        dist = np.linalg.norm(outside - x, axis=1)
        assert dist.min() >= R * (1 - 1e-12), (x, R, dist.min())


@pytest.mark.parametrize("dim", [2, 3])
def test_csg_closest_point_lies_on_the_boundary(orc, dim):
    """Near the boundary (away from creases) x - sdf grad sdf lands on the zero set."""
    prob = W.csg_laplace_problem(dim)
    inside, X, d = _inside_points(orc, prob, 40000, seed=2)
    near = X[(d > 0) & (d < 2e-3)]
    assert len(near) > 20
    on = 0
    for x in near:
        _, xb = orc.distance(prob, x)
        if abs(orc.distance(prob, xb)[0]) <= 1e-9:
            on += 1
    assert on >= 0.95 * len(near)


@pytest.mark.parametrize("dim", [2, 3])
def test_csg_walk_matches_harmonic_boundary_data(orc, dim):
    """Laplace on a CSG scene with harmonic g: u = g (Kakutani), within 4 standard errors."""
    from tests.stats_util import four_se_rule
    prob = W.csg_laplace_problem(dim)
    inside, _, _ = _inside_points(orc, prob, 20000, seed=3, margin=0.02)
    pts = inside[:16].T.copy()
    sb = orc.sigma_bar(prob)[0]
    acc, st = orc.solve(prob, pts, 3000, seed=1, eps=1e-4, sigma_bar=sb)
    m, v, se = orc.finalize(acc)
    ok, nout, mz = four_se_rule((m - W.csg_laplace_exact(dim, pts)) / se)
    assert ok and st["capped"] == 0


def test_csg_variable_coefficients_manufactured(orc):
    from tests.stats_util import four_se_rule
    prob = W.csg_variable_problem()
    inside, _, _ = _inside_points(orc, prob, 20000, seed=4, margin=0.02)
    pts = inside[:12].T.copy()
    sb = orc.sigma_bar(prob)[0]
    acc, st = orc.solve(prob, pts, 3000, seed=2, eps=1e-4, sigma_bar=sb)
    m, v, se = orc.finalize(acc)
    ok, nout, mz = four_se_rule((m - W.cube3d_exact(*pts)) / se)
    assert ok
