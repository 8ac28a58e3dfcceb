"""Pins of the finite-difference references used by other tests (tests/fd_reference.py).

* The 2D solver converges at second order to a closed-form solution of eq. 1
  (the square2d manufactured problem: variable alpha and sigma).
* The 3D discrete adjoint equals central differences of the discrete functional.
* The 3D solution and gradient settle as the grid is refined (grids aligned with
  the sigma grid's nodes).
"""
import numpy as np

import workloads as W
from tests.fd_reference import fd_cube_sigma_gradient, fd_solve_square


def test_square_solver_second_order_on_a_closed_form():
    c = {
        "alpha": lambda x, y: 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y),
        "grad_phi": lambda x, y: (0.0 * x, 0.0 * y),
        "sigma": lambda x, y: 2.0 + np.sin(3.0 * x + y),
        "g": lambda x, y: W.square2d_exact(x, y),
    }
    # f of eq. 1 for u = sin(pi x) cosh(y) with this alpha and sigma, written out
    def f(x, y):
        u = np.sin(np.pi * x) * np.cosh(y)
        ux, uy = np.pi * np.cos(np.pi * x) * np.cosh(y), np.sin(np.pi * x) * np.sinh(y)
        lap = -np.pi ** 2 * u + u
        a = c["alpha"](x, y)
        ax = np.pi * np.cos(2 * np.pi * x) * np.cos(2 * np.pi * y)
        ay = -np.pi * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
        return -(a * lap + ax * ux + ay * uy) + c["sigma"](x, y) * u
    c["f"] = f
    errs = []
    for n in (32, 64):
        u = fd_solve_square(c, n)
        xs = np.arange(n + 1) / n
        X, Y = np.meshgrid(xs, xs, indexing="ij")
        errs.append(np.abs(u - W.square2d_exact(X, Y)).max())
    assert errs[1] < 1e-3 and 3.5 < errs[0] / errs[1] < 4.5, errs


def _inverse_setup(k=24):
    sig = W.inverse_sigma_grid()
    alpha = W.inverse_alpha_grid()
    pts = W.inverse_sensors(k, seed=4).astype(np.float64)
    w = np.random.default_rng(0).normal(size=k)
    return sig, alpha, pts, w, (lambda x, y, z: np.ones_like(x)), (lambda x, y, z: 1 + x * y + z)


def test_cube_discrete_adjoint_equals_differences():
    sig, alpha, pts, w, f, g = _inverse_setup()
    n = 20
    _, grad = fd_cube_sigma_gradient(alpha, sig, f, g, n, pts, w)
    nodes = np.argsort(-np.abs(grad))[:3]
    for node in nodes:
        vals = []
        for s in (1, -1):
            s2 = sig.astype(np.float64).reshape(-1).copy()
            s2[node] += s * 1e-3
            vals.append(w @ fd_cube_sigma_gradient(alpha, s2.reshape(sig.shape), f, g, n, pts, w)[0])
        fd = (vals[0] - vals[1]) / 2e-3
        assert abs(grad[node] - fd) <= 1e-6 * abs(fd), (node, grad[node], fd)


def test_cube_refinement_settles():
    sig, alpha, pts, w, f, g = _inverse_setup()
    u31, g31 = fd_cube_sigma_gradient(alpha, sig, f, g, 31, pts, w)
    u62, g62 = fd_cube_sigma_gradient(alpha, sig, f, g, 62, pts, w)
    assert np.abs(u31 - u62).max() < 2e-3
    assert np.linalg.norm(g31 - g62) / np.linalg.norm(g62) < 0.15
