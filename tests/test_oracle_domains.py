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
