"""End-to-end pins of the oracle's delta-tracking walk against exact solutions.

Harmonic boundary data on a disk and a ball (Kakutani's principle, Sec. 2.4),
constant screening with a known solution (Sec. 2.3), and the manufactured
variable-coefficient problems (eq. 1 with alpha, sigma and a conservative drift
chosen so that u is known).  Any sigma_bar > 0 leaves the estimator unbiased
(Sec. 5.1), so estimates at sigma_bar and 2 sigma_bar must agree.
"""
import numpy as np
import pytest

import workloads as W
from tests.stats_util import combined_z, four_se_rule


def _run(orc, prob, pts, walks, eps, sb=None, seed=0, offset=0):
    if sb is None:
        sb = orc.sigma_bar(prob)[0]
    acc, st = orc.solve(prob, pts, walks, seed=seed, eps=eps, sigma_bar=sb, walk_offset=offset)
    m, v, se = orc.finalize(acc)
    assert st["capped"] == 0 and st["nonfinite"] == 0
    return m, se, st


CASES = {
    "laplace_disk": (W.laplace_disk_problem, lambda p: W.laplace_disk_exact(*p),
                     lambda: W.uniform_in_ball(2, 12, [0, 0], 1.0, seed=1, margin=0.05), 4000, 1e-4),
    "laplace_ball": (W.laplace_ball_problem, lambda p: W.laplace_ball_exact(*p),
                     lambda: W.uniform_in_ball(3, 12, [0, 0, 0], 1.0, seed=2, margin=0.05), 3000, 1e-4),
    "screened_square": (W.screened_square_problem, lambda p: W.screened_square_exact(*p),
                        lambda: W.uniform_in_box(2, 12, 0.05, 0.95, seed=3), 4000, 1e-4),
    "screened_ball": (W.screened_ball_problem, lambda p: W.screened_ball_exact(9.0, *p),
                      lambda: W.uniform_in_ball(3, 12, [0, 0, 0], 1.0, seed=4, margin=0.05), 3000, 1e-4),
    "square2d": (W.square2d_problem, lambda p: W.square2d_exact(*p),
                 lambda: W.cell_centres(2, 32)[:, W.seeded_subset(1024, 16, 5)], 6000, 1e-3),
    "cube3d": (W.cube3d_problem, lambda p: W.cube3d_exact(*p),
               lambda: W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 10, 6)], 3000, 1e-4),
}


@pytest.mark.parametrize("name", list(CASES))
def test_walk_matches_exact_solution(orc, name):
    mk, exact, ptsf, walks, eps = CASES[name]
    prob = mk()
    pts = ptsf()
    m, se, st = _run(orc, prob, pts, walks, eps)
    u = exact(pts.astype(np.float64))
    z = (m - u) / se
    ok, nout, mz = four_se_rule(z)
    assert ok, (name, z)
    assert st["steps"] > st["walks"]


def test_sigma_bar_invariance(orc):
    prob = W.square2d_problem()
    pts = W.cell_centres(2, 32)[:, W.seeded_subset(1024, 12, 7)]
    sb = orc.sigma_bar(prob)[0]
    m1, se1, st1 = _run(orc, prob, pts, 3000, 1e-3, sb=sb, seed=1)
    m2, se2, st2 = _run(orc, prob, pts, 3000, 1e-3, sb=2 * sb, seed=2)
    ok, _, _ = four_se_rule(combined_z(m1, se1, m2, se2))
    assert ok
    # a larger bound makes more null events: more steps per walk (Sec. 5.2, Fig. 12)
    assert st2["steps"] > 1.1 * st1["steps"]


def test_walk_ids_continue_streams(orc):
    """Walk j of a run at offset o is walk o + j of a run at offset 0 (bit for bit)."""
    prob = W.cube3d_problem()
    pts = W.cell_centres(3, 64)[:, :3]
    sb = orc.sigma_bar(prob)[0]
    a, sa = orc.walks(prob, pts, 8, seed=11, eps=1e-4, sigma_bar=sb)
    b, sb_ = orc.walks(prob, pts, 4, seed=11, eps=1e-4, sigma_bar=sb, walk_offset=4)
    assert np.array_equal(a[:, 4:], b)
    assert np.array_equal(sa[:, 4:], sb_)
    c, _ = orc.walks(prob, pts, 8, seed=12, eps=1e-4, sigma_bar=sb)
    assert not np.array_equal(a, c)


def test_points_in_shell_return_boundary_value(orc):
    """A point already within eps of the boundary returns g(xbar) exactly (Alg. 1)."""
    prob = W.square2d_problem()
    pts = np.array([[0.5, 1e-4, 0.3], [0.9995, 0.5, 1 - 2e-4]], dtype=np.float32)
    sb = orc.sigma_bar(prob)[0]
    uh, steps = orc.walks(prob, pts, 5, seed=0, eps=1e-3, sigma_bar=sb)
    assert np.all(steps == 0)
    for i in range(3):
        d, xb = orc.distance(prob, pts[:, i].astype(np.float64))
        want = W.square2d_exact(*xb)
        assert np.allclose(uh[i], want, rtol=1e-12, atol=1e-14)


def test_step_cap_is_reported(orc):
    prob = W.square2d_problem()
    pts = W.cell_centres(2, 4)
    sb = orc.sigma_bar(prob)[0]
    _, st = orc.solve(prob, pts, 50, seed=0, eps=1e-3, sigma_bar=sb, max_steps=2)
    assert st["capped"] > 0
    assert st["steps"] <= 2 * st["walks"]


# ---------------------------------------------------------------------------
# weight window (Sec. 6)
# ---------------------------------------------------------------------------
def test_window_off_equals_plain_walk(orc):
    prob = W.cube3d_problem()
    sb = orc.sigma_bar(prob)[0]
    x = W.cell_centres(3, 64)[:, 1234].astype(np.float64)
    for j in range(20):
        u0, k0, _ = orc.walk(prob, x, 7, j, 5, 1e-4, sb)
        u1, k1, _ = orc.walk_ww(prob, x, 7, j, 5, 1e-4, sb, 0.0, 1.0)
        assert u0 == u1 and k0 == k1


@pytest.mark.parametrize("depth", [8, 1])
def test_window_unbiased_exact_solution(orc, depth):
    prob = W.hifreq_alpha_problem()
    sb = orc.sigma_bar(prob)[0]
    pts = W.cell_centres(2, 8)[:, ::5]
    acc, st = orc.solve_ww(prob, pts, 1500, seed=3, eps=1e-3, sigma_bar=sb, ww_lo=0.5, ww_hi=1.5, depth=depth)
    m, v, se = orc.finalize(acc)
    ok, _, _ = four_se_rule((m - W.hifreq_alpha_exact(*pts.astype(np.float64))) / se)
    assert ok
    assert st["capped"] == 0 and st["nonfinite"] == 0


def test_window_reduces_variance_high_frequency_alpha(orc):
    """Sec. 6 (weight-window figure): with a high-frequency alpha the plain estimator's
    error is dominated by rare walks of huge weight; the window cuts the mean squared
    error against the exact solution (here more than 3x) at fewer steps per walk."""
    prob = W.hifreq_alpha_problem()
    sb = orc.sigma_bar(prob)[0]
    pts = W.cell_centres(2, 8)
    exact = W.hifreq_alpha_exact(*pts.astype(np.float64))
    a0, s0 = orc.solve(prob, pts, 1500, seed=5, eps=1e-3, sigma_bar=sb)
    a1, s1 = orc.solve_ww(prob, pts, 1500, seed=5, eps=1e-3, sigma_bar=sb, ww_lo=0.5, ww_hi=1.5)
    mse0 = np.mean((orc.finalize(a0)[0] - exact) ** 2)
    mse1 = np.mean((orc.finalize(a1)[0] - exact) ** 2)
    assert mse1 < mse0 / 3
    assert s1["steps"] / s1["walks"] < s0["steps"] / s0["walks"]


# ---------------------------------------------------------------------------
# a problem without a closed-form solution: fine finite-difference reference
# ---------------------------------------------------------------------------
def test_walk_matches_finite_difference_solve(orc):
    """Variable alpha, conservative drift, variable sigma, a source and non-harmonic g on the
    unit square (eq. 1): the walk's mean agrees with a second-order finite-difference solve
    (N = 256, discretisation error ~1e-5, far below the standard errors)."""
    from tests.fd_reference import fd_reference_at
    prob = W.fd_square_problem()
    c = W.fd_square_coefficients()
    # the numpy coefficients are the problem's (checked at a few points)
    for x in np.random.default_rng(0).uniform(0, 1, size=(5, 2)):
        assert np.isclose(orc.field_eval(prob, "alpha", x)[0], c["alpha"](*x), rtol=1e-12)
        assert np.allclose(orc.field_eval(prob, "phi", x)[1], c["grad_phi"](*x), rtol=1e-12)
        assert np.isclose(orc.field_eval(prob, "sigma", x)[0], c["sigma"](*x), rtol=1e-12)
        assert np.isclose(orc.field_eval(prob, "f", x)[0], c["f"](*x), rtol=1e-12)
        assert np.isclose(orc.field_eval(prob, "g", x)[0], c["g"](*x), rtol=1e-12)
    g = np.array([0.125, 0.375, 0.625, 0.875])
    pts = np.array(np.meshgrid(g, g, indexing="ij")).reshape(2, -1)
    want = fd_reference_at(c, pts, n=256)
    m, se, st = _run(orc, prob, pts, 6000, 1e-4)
    ok, nout, mz = four_se_rule((m - want) / se)
    assert ok, ((m - want) / se)
