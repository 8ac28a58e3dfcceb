"""Pins of the oracle's mesh boundary: its BVH against brute force over all triangles,
its point-triangle closest point against dense sampling of the triangle, and the walk on
a mesh domain against a manufactured solution (exact on any domain)."""
import numpy as np
import pytest

import workloads as W
from tests.stats_util import four_se_rule


@pytest.fixture(scope="module")
def mesh7():
    return W.mesh_manufactured_problem(level=7)


def test_bvh_equals_brute_force(orc, mesh7):
    pk = orc.pack(mesh7)
    rng = np.random.default_rng(0)
    pts = np.concatenate([rng.uniform(-0.95, 0.95, size=(40, 3)), rng.normal(size=(10, 3)) * 0.6])
    for x in pts:
        d, xb = orc.distance(mesh7, x, packed=pk)
        db, xbb = orc.mesh_distance_brute(mesh7, x, packed=pk)
        assert d == db
        # ties between triangles that share the closest edge or vertex give the same point up to rounding
        assert np.allclose(xb, xbb, rtol=0, atol=1e-12)


def test_closest_point_on_triangle_dense_sampling(orc):
    rng = np.random.default_rng(1)
    for _ in range(30):
        tri_v = rng.normal(size=(3, 3)).astype(np.float32)
        prob = W.problem(3, W.mesh_domain(tri_v, np.array([[0, 1, 2]], dtype=np.int32)), W.const(1), W.zero(),
                         W.zero(), W.zero())
        x = rng.normal(size=3) * 1.5
        d, xb = orc.mesh_distance_brute(prob, x)
        # dense barycentric sampling of the triangle bounds the distance from above
        s = np.linspace(0, 1, 201)
        a, b = np.meshgrid(s, s)
        m = a + b <= 1
        P = (tri_v[0][None, :] * (1 - a[m] - b[m])[:, None] + tri_v[1][None, :] * a[m][:, None]
             + tri_v[2][None, :] * b[m][:, None])
        dense = np.linalg.norm(P - x, axis=1).min()
        assert d <= dense + 1e-12
        assert d >= dense - 0.02 * np.linalg.norm(tri_v[1] - tri_v[0]) - 0.02 * np.linalg.norm(tri_v[2] - tri_v[0])
        # the closest point is on the triangle at distance d
        assert np.linalg.norm(xb - x) == pytest.approx(d, rel=1e-12, abs=1e-12)
        M = np.stack([tri_v[1] - tri_v[0], tri_v[2] - tri_v[0]], 1).astype(np.float64)
        bary, *_ = np.linalg.lstsq(M, xb - tri_v[0], rcond=None)
        assert np.allclose(M @ bary, xb - tri_v[0], atol=1e-9)
        assert bary.min() >= -1e-6 and bary.sum() <= 1 + 1e-6


def test_walk_on_mesh_matches_exact_solution(orc):
    prob = W.mesh_manufactured_problem(level=5)
    pts = W.mesh_interior_points(10, seed=5)
    sb = orc.sigma_bar(prob, 48)[0]
    acc, st = orc.solve(prob, pts, 3000, seed=0, eps=1e-4, sigma_bar=sb)
    m, v, se = orc.finalize(acc)
    exact = W.cube3d_exact(*pts.astype(np.float64))
    ok, nout, mz = four_se_rule((m - exact) / se)
    assert ok, ((m - exact) / se)
    assert st["capped"] == 0 and st["nonfinite"] == 0


def test_distance_grid_radius_is_a_lower_bound(orc):
    """With a distance grid the radius is max_c (d(c) - |x - c|) over the cell corners (the
    distance is 1-Lipschitz): never above the brute-force distance, exact below the threshold."""
    pg = W.mesh_manufactured_problem(level=4, dist_grid=24)
    pe = W.mesh_manufactured_problem(level=4)
    X = W.mesh_interior_points(400, 9).T.astype(np.float64)
    ratios = []
    for x in X:
        brute, _ = orc.mesh_distance_brute(pe, x)
        dg, _ = orc.distance(pg, x)
        assert dg <= brute * (1 + 1e-12) + 1e-15
        ratios.append(dg / brute)
    ratios = np.array(ratios)
    assert ratios.mean() > 0.9 and (ratios == 1.0).any()


def test_distance_grid_walk_matches_exact_solution(orc):
    """Smaller balls leave the estimator unbiased: the manufactured solution within 4 SE."""
    pg = W.mesh_manufactured_problem(level=5, dist_grid=48)
    pts = W.mesh_interior_points(16, 7)
    sb = orc.sigma_bar(pg)[0]
    acc, st = orc.solve(pg, pts, 3000, seed=5, eps=1e-4, sigma_bar=sb)
    m, v, se = orc.finalize(acc)
    exact = W.cube3d_exact(*pts.astype(np.float64))
    ok, nout, mz = four_se_rule((m - exact) / se)
    assert ok and st["capped"] == 0
