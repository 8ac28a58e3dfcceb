"""Pins of the oracle's coefficient fields and of the PDE transformation.

Independent references: sympy expressions of the same closed forms, sympy's
derivation of the manufactured source from eq. 1, and the substitution check
that U = e^gamma u solves Lap U - sigma' U = -f' (Sec. 4.1, App. A).  The last
one also fixes the sign of the right-hand side of the transformed equation,
which the paper prints as +f' in eq. 8 but whose derivation (App. A) gives -f'.
"""
import numpy as np
import pytest
import sympy as sp

import workloads as W

X = sp.symbols("x0 x1 x2", real=True)
_H = {
    W.ONE: lambda t: sp.Integer(1), W.SIN: sp.sin, W.COS: sp.cos, W.EXP: sp.exp,
    W.SINH: sp.sinh, W.COSH: sp.cosh, W.LIN: lambda t: t, W.QUAD: lambda t: t ** 2,
}


def sym_field(fd, dim):
    if fd["kind"] == "zero":
        return sp.Integer(0)
    if fd["kind"] == "const":
        return sp.Float(fd["value"])
    assert fd["kind"] == "sst"
    e = sp.Integer(0)
    for t in fd["terms"]:
        prod = sp.Float(t["c"])
        for d in range(dim):
            ty, k, ph = t["atoms"][d]
            prod *= _H[ty](sp.Float(k) * X[d] + sp.Float(ph))
        e += prod
    return e


def grad(e, dim):
    return [sp.diff(e, X[d]) for d in range(dim)]


def lap(e, dim):
    return sum(sp.diff(e, X[d], 2) for d in range(dim))


PROBLEMS = {
    "square2d": W.square2d_problem(),
    "cube3d": W.cube3d_problem(),
    "screened_square": W.screened_square_problem(),
    "screened_ball": W.screened_ball_problem(),
    "laplace_ball": W.laplace_ball_problem(),
}


def _points(dim, n=6, seed=3):
    return np.random.default_rng(seed).uniform(0.05, 0.95, size=(n, dim))


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_sst_value_grad_lap(orc, name):
    prob = PROBLEMS[name]
    dim = prob["dim"]
    pk = orc.pack(prob)
    for fname in ("alpha", "phi", "sigma", "um", "g"):
        e = sym_field(prob[fname], dim)
        ge, le = grad(e, dim), lap(e, dim)
        for x in _points(dim):
            sub = {X[d]: x[d] for d in range(dim)}
            v, g, l_ = orc.field_eval(prob, fname, x, packed=pk)
            assert v == pytest.approx(float(e.subs(sub)), rel=1e-12, abs=1e-12)
            for d in range(dim):
                assert g[d] == pytest.approx(float(ge[d].subs(sub)), rel=1e-12, abs=1e-12)
            assert l_ == pytest.approx(float(le.subs(sub)), rel=1e-12, abs=1e-11)


def _sym_problem(prob):
    dim = prob["dim"]
    u = sym_field(prob["um"], dim)
    a = sym_field(prob["alpha"], dim)
    ph = sym_field(prob["phi"], dim)
    s = sym_field(prob["sigma"], dim)
    omega = [a * gd for gd in grad(ph, dim)]
    # eq. 1: div(alpha grad u) + omega . grad u - sigma u = -f
    div = sum(sp.diff(a * sp.diff(u, X[d]), X[d]) for d in range(dim))
    f = -(div + sum(omega[d] * sp.diff(u, X[d]) for d in range(dim)) - s * u)
    return dim, u, a, ph, s, f


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_manufactured_source_matches_eq1(orc, name):
    prob = PROBLEMS[name]
    dim, u, a, ph, s, f = _sym_problem(prob)
    if prob["f"]["kind"] != "manufactured":
        pytest.skip("source given directly")
    pk = orc.pack(prob)
    for x in _points(dim):
        sub = {X[d]: x[d] for d in range(dim)}
        v, _, _ = orc.field_eval(prob, "f", x, packed=pk)
        assert v == pytest.approx(float(f.subs(sub)), rel=1e-11, abs=1e-11)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_transformed_equation_residual(orc, name):
    """U = e^gamma u with the oracle's gamma, sigma', f' satisfies Lap U - sigma' U + f' = 0."""
    prob = PROBLEMS[name]
    dim, u, a, ph, s, f = _sym_problem(prob)
    gam = sp.log(a) / 2 + ph / 2
    U = sp.exp(gam) * u
    LU = lap(U, dim)
    pk = orc.pack(prob)
    for x in _points(dim):
        sub = {X[d]: x[d] for d in range(dim)}
        g_o, sp_o, fp_o, f_o, a_o = orc.coeffs(prob, x, packed=pk)
        assert g_o == pytest.approx(float(gam.subs(sub)), rel=1e-12, abs=1e-12)
        Uv, LUv = float(U.subs(sub)), float(LU.subs(sub))
        scale = abs(LUv) + abs(sp_o * Uv) + abs(fp_o) + 1e-12
        assert abs(LUv - sp_o * Uv + fp_o) / scale < 1e-10


def test_paper_sigma_prime_without_drift(orc):
    """With omega = 0, sigma' reduces to the printed sigma/alpha + (Lap a/a - |grad ln a|^2/2)/2."""
    prob = W.square2d_problem()
    dim = 2
    a = sym_field(prob["alpha"], dim)
    s = sym_field(prob["sigma"], dim)
    gl = grad(sp.log(a), dim)
    printed = s / a + sp.Rational(1, 2) * (lap(a, dim) / a - sum(g * g for g in gl) / 2)
    pk = orc.pack(prob)
    for x in _points(dim):
        sub = {X[d]: x[d] for d in range(dim)}
        assert orc.coeffs(prob, x, packed=pk)[1] == pytest.approx(float(printed.subs(sub)),
                                                                  rel=1e-11)


def test_grid_fields_reproduce_linear(orc):
    """Multilinear and cubic B-spline grids reproduce a linear function inside the grid."""
    res = (9, 7, 5)
    lo, hi = (-1.0, 0.0, 0.5), (1.0, 2.0, 1.5)
    ax = [np.linspace(lo[d], hi[d], res[d]) for d in range(3)]
    zz, yy, xx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    data = (0.5 + 2.0 * xx - 1.5 * yy + 0.25 * zz).astype(np.float32)
    for kind in ("grid_linear", "grid_bspline"):
        fd = {"kind": kind, "res": res, "lo": lo, "hi": hi, "data": data}
        prob = W.problem(3, W.box(lo, hi), fd, W.zero(), W.zero(), W.zero())
        rng = np.random.default_rng(1)
        for _ in range(20):
            # stay one cell away from the faces: the B-spline's clamped control points
            # bend a linear function there
            h = [(hi[d] - lo[d]) / (res[d] - 1) for d in range(3)]
            x = np.array([rng.uniform(lo[d] + 1.01 * h[d], hi[d] - 1.01 * h[d]) for d in range(3)])
            v, g, l_ = orc.field_eval(prob, "alpha", x)
            assert v == pytest.approx(0.5 + 2.0 * x[0] - 1.5 * x[1] + 0.25 * x[2], abs=1e-5)
            assert g == pytest.approx([2.0, -1.5, 0.25], abs=1e-4)
            assert l_ == pytest.approx(0.0, abs=1e-3)


def test_bspline_derivatives_match_differences(orc):
    rng = np.random.default_rng(2)
    res = (6, 6, 6)
    data = rng.uniform(0.5, 2.0, size=res).astype(np.float32)
    fd = {"kind": "grid_bspline", "res": res, "lo": (0, 0, 0), "hi": (1, 1, 1), "data": data}
    prob = W.problem(3, W.box((0, 0, 0), (1, 1, 1)), fd, W.zero(), W.zero(), W.zero())
    h = 1e-4
    for _ in range(10):
        x = rng.uniform(0.05, 0.95, size=3)
        v, g, l_ = orc.field_eval(prob, "alpha", x)
        lap_fd = 0.0
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            vp = orc.field_eval(prob, "alpha", x + e)[0]
            vm = orc.field_eval(prob, "alpha", x - e)[0]
            assert g[d] == pytest.approx((vp - vm) / (2 * h), rel=1e-5, abs=1e-6)
            lap_fd += (vp - 2 * v + vm) / (h * h)
        assert l_ == pytest.approx(lap_fd, rel=1e-3, abs=1e-3)


def _cardinal_bspline_field(data, lo, hi, x):
    """Value, gradient and Laplacian of sum_j c_j N(s - j + 2) per axis, N the cubic
    basis element on the knots 0..4 from scipy's Cox-de Boor recursion, s the point in
    node units, control indices clamped to the grid (array index [z, y, x])."""
    from scipy.interpolate import BSpline
    N = BSpline.basis_element(np.arange(5.0), extrapolate=False)
    dN, d2N = N.derivative(1), N.derivative(2)
    res = data.shape[::-1]
    h = [(hi[d] - lo[d]) / (res[d] - 1) for d in range(3)]
    s = [(x[d] - lo[d]) / h[d] for d in range(3)]
    base = [int(np.floor(s[d])) - 1 for d in range(3)]
    w = [[], [], []]
    for d in range(3):
        for a in range(4):
            t = s[d] - (base[d] + a) + 2.0
            w[d].append((float(N(t)), float(dN(t)) / h[d], float(d2N(t)) / h[d] ** 2))
    v, g, lap = 0.0, np.zeros(3), 0.0
    for c in range(4):
        for b in range(4):
            for a in range(4):
                i = [min(max(base[0] + a, 0), res[0] - 1), min(max(base[1] + b, 0), res[1] - 1),
                     min(max(base[2] + c, 0), res[2] - 1)]
                cv = float(data[i[2], i[1], i[0]])
                wx, wy, wz = w[0][a], w[1][b], w[2][c]
                v += cv * wx[0] * wy[0] * wz[0]
                g += cv * np.array([wx[1] * wy[0] * wz[0], wx[0] * wy[1] * wz[0], wx[0] * wy[0] * wz[1]])
                lap += cv * (wx[2] * wy[0] * wz[0] + wx[0] * wy[2] * wz[0] + wx[0] * wy[0] * wz[2])
    return v, g, lap


def test_bspline_grid_is_the_cardinal_cubic_bspline(orc):
    """The B-spline grid field (reading R6: node values as control points of a uniform
    cubic B-spline, C^2) equals the textbook cardinal cubic B-spline built from scipy's
    Cox-de Boor basis element: value, gradient and Laplacian, inside the grid and near
    its faces (clamped control indices).  An interpolating cubic (Catmull-Rom) or a
    wrong basis that still sums to one fails this."""
    rng = np.random.default_rng(11)
    res = (7, 6, 5)
    lo, hi = (-0.5, 0.0, 1.0), (1.0, 2.0, 2.0)
    data = rng.uniform(0.5, 2.0, size=res[::-1]).astype(np.float32)
    fd = {"kind": "grid_bspline", "res": res, "lo": lo, "hi": hi, "data": data}
    prob = W.problem(3, W.box(lo, hi), fd, W.zero(), W.zero(), W.zero())
    for _ in range(40):
        x = np.array([rng.uniform(lo[d], hi[d]) for d in range(3)])
        v, g, l_ = orc.field_eval(prob, "alpha", x)
        rv, rg, rl = _cardinal_bspline_field(data, lo, hi, x)
        assert v == pytest.approx(rv, rel=1e-12, abs=1e-12)
        assert np.asarray(g) == pytest.approx(rg, rel=1e-10, abs=1e-10)
        assert l_ == pytest.approx(rl, rel=1e-9, abs=1e-9)


def test_bspline_grid_node_identity_and_c2_faces(orc):
    """At an interior node the cubic B-spline takes (c_{i-1} + 4 c_i + c_{i+1}) / 6 along
    each axis (a tensor product of that stencil), not the node value; across a cell face
    the value, gradient and Laplacian are continuous (C^2, which sigma' needs)."""
    rng = np.random.default_rng(12)
    res = (6, 6, 6)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    data = rng.uniform(0.5, 2.0, size=res).astype(np.float64)
    fd = {"kind": "grid_bspline", "res": res, "lo": lo, "hi": hi, "data": data.astype(np.float32)}
    prob = W.problem(3, W.box(lo, hi), fd, W.zero(), W.zero(), W.zero())
    c = data.astype(np.float32).astype(np.float64)
    st = np.array([1.0, 4.0, 1.0]) / 6.0
    for (i, j, k) in [(1, 1, 1), (2, 3, 4), (4, 2, 3)]:
        x = np.array([i, j, k], dtype=np.float64) / 5.0
        want = np.einsum("a,b,c,cba->", st, st, st, c[k - 1:k + 2, j - 1:j + 2, i - 1:i + 2])
        assert orc.field_eval(prob, "alpha", x)[0] == pytest.approx(want, rel=1e-12)
    # continuity across the face x = 0.4 (a node plane) at random (y, z)
    delta = 1e-7
    for _ in range(10):
        y, z = rng.uniform(0.05, 0.95, size=2)
        a = orc.field_eval(prob, "alpha", np.array([0.4 - delta, y, z]))
        b = orc.field_eval(prob, "alpha", np.array([0.4 + delta, y, z]))
        assert a[0] == pytest.approx(b[0], abs=1e-5)
        assert np.asarray(a[1]) == pytest.approx(np.asarray(b[1]), abs=1e-4)
        assert a[2] == pytest.approx(b[2], abs=2e-3)
