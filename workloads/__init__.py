"""Seeded synthetic inputs for delta-tracking walk on spheres.

This module only *describes* problems and generates inputs: domains, the
closed-form coefficient families, the evaluation points and the seeds.  It
holds none of the method's arithmetic, so both the CUDA path and the CPU
oracle can take their inputs from here without sharing any computation.

A problem is a plain dict::

    {"dim": 2|3,
     "domain": {"kind": "box"|"ball"|"annulus"|"rounded_box", "p": [..16 floats]},
     "alpha": field, "phi": field, "sigma": field, "f": field, "g": field,
     "um": field}

and a field is ``{"kind": "zero"|"const"|"sst"|"manufactured"|"grid_linear"|
"grid_bspline", ...}``.  An ``sst`` field is a sum of separable terms
``c * prod_i h_i(k_i x_i + phi_i)`` with ``h`` one of ONE, SIN, COS, EXP,
SINH, COSH, LIN (t) and QUAD (t^2).  ``manufactured`` asks for the source
``f = -div(alpha grad um) - omega . grad um + sigma um`` of the PDE (Sec. 3,
eq. 1) at the given ``um``, with ``omega = alpha grad phi``.

The manufactured workloads are the paper's PDE with coefficients chosen so the
exact solution is known (Sec. 3 eq. 1; App. A for the drift).
"""
from __future__ import annotations

import math

import numpy as np

ONE, SIN, COS, EXP, SINH, COSH, LIN, QUAD = range(8)
ATOM_NAMES = ["ONE", "SIN", "COS", "EXP", "SINH", "COSH", "LIN", "QUAD"]

PI = math.pi


def term(c, *atoms):
    """One separable term: c * prod_i h_i(k_i x_i + phi_i); atoms are (type, k, phi)."""
    a = [tuple(x) if x is not None else (ONE, 0.0, 0.0) for x in atoms]
    while len(a) < 3:
        a.append((ONE, 0.0, 0.0))
    return {"c": float(c), "atoms": [(int(t), float(k), float(p)) for t, k, p in a]}


def sst(*terms):
    return {"kind": "sst", "terms": list(terms)}


def const(v):
    return {"kind": "const", "value": float(v)}


def zero():
    return {"kind": "zero"}


def manufactured():
    return {"kind": "manufactured"}


def box(lo, hi):
    p = [0.0] * 16
    for i, v in enumerate(lo):
        p[i] = float(v)
    for i, v in enumerate(hi):
        p[3 + i] = float(v)
    return {"kind": "box", "p": p}


def ball(centre, radius):
    p = [0.0] * 16
    for i, v in enumerate(centre):
        p[i] = float(v)
    p[3] = float(radius)
    return {"kind": "ball", "p": p}


def annulus(centre, r_in, r_out):
    p = [0.0] * 16
    for i, v in enumerate(centre):
        p[i] = float(v)
    p[3] = float(r_in)
    p[4] = float(r_out)
    return {"kind": "annulus", "p": p}


def rounded_box(centre, half, corner):
    p = [0.0] * 16
    for i, v in enumerate(centre):
        p[i] = float(v)
    for i, v in enumerate(half):
        p[3 + i] = float(v)
    p[6] = float(corner)
    return {"kind": "rounded_box", "p": p}


def csg(lo, hi, *nodes):
    """Signed-distance CSG domain: nodes are (primitive, op, params) with primitive one of
    sphere, box, capsule, torus, halfspace and op one of union, intersect, subtract (the
    first node's op is ignored); lo, hi bound the domain."""
    p = [0.0] * 16
    for i, v in enumerate(lo):
        p[i] = float(v)
    for i, v in enumerate(hi):
        p[3 + i] = float(v)
    out = []
    for prim, op, prm in nodes:
        q = [float(v) for v in prm] + [0.0] * (8 - len(prm))
        out.append((prim, op, q))
    return {"kind": "csg", "p": p, "nodes": out}


def problem(dim, domain, alpha, sigma, f, g, phi=None, um=None, omega=None, drift_bound=0.0):
    """omega: an extra drift vector field (a list of dim fields), added to alpha grad(phi);
    drift_bound: 0 or an upper bound of |omega / alpha| over the domain."""
    om = list(omega) if omega is not None else []
    om += [zero()] * (3 - len(om))
    return {
        "drift_bound": float(drift_bound),
        "dim": int(dim),
        "domain": domain,
        "alpha": alpha,
        "phi": phi if phi is not None else zero(),
        "sigma": sigma,
        "f": f,
        "g": g,
        "um": um if um is not None else zero(),
        "omega": om,
    }


# ---------------------------------------------------------------------------
# Workload 1: 2D unit square, u = sin(pi x) cosh(y),
#   alpha = 1 + 0.5 sin(2 pi x) cos(2 pi y), sigma = 2 + sin(3x + y), omega = 0,
#   f derived from eq. 1, g = u; eps = 1e-3; 32 x 32 cell centres x 256 walks.
# ---------------------------------------------------------------------------
def square2d_problem():
    u = sst(term(1.0, (SIN, PI, 0.0), (COSH, 1.0, 0.0)))
    alpha = sst(term(1.0), term(0.5, (SIN, 2 * PI, 0.0), (COS, 2 * PI, 0.0)))
    # sin(3x + y) = sin(3x) cos(y) + cos(3x) sin(y)
    sigma = sst(term(2.0), term(1.0, (SIN, 3.0, 0.0), (COS, 1.0, 0.0)),
                term(1.0, (COS, 3.0, 0.0), (SIN, 1.0, 0.0)))
    return problem(2, box([0, 0], [1, 1]), alpha, sigma, manufactured(), u, um=u)


def square2d_exact(x, y):
    return np.sin(np.pi * x) * np.cosh(y)


def square2d_exact_grad(x, y):
    """grad u of square2d_exact, shape [2, ...]."""
    return np.array([np.pi * np.cos(np.pi * x) * np.cosh(y), np.sin(np.pi * x) * np.sinh(y)])


SQUARE2D = {"name": "square2d_manufactured", "eps": 1e-3, "grid": 32, "walks": 256,
            "seed": 0}


# ---------------------------------------------------------------------------
# Workload 2: 3D unit cube with a conservative drift,
#   u = exp(0.5 x) sin(pi y) cos(pi z), alpha = 1 + 0.3 |x|^2, sigma = 1 + x y,
#   omega = alpha grad(Phi), Phi = x sin(2 pi y) + sin(2 pi z)/(2 pi) + 0.5 z,
#   so omega/alpha = (sin 2pi y, 2pi x cos 2pi y, cos 2pi z + 0.5);
#   eps = 1e-4; 64^3 cell centres x 1024 walks.
# The paper removes a drift exactly only when omega/alpha is a gradient
# (App. A), so the drift is given through its potential Phi.
# ---------------------------------------------------------------------------
def cube3d_problem():
    u = sst(term(1.0, (EXP, 0.5, 0.0), (SIN, PI, 0.0), (COS, PI, 0.0)))
    alpha = sst(term(1.0), term(0.3, (QUAD, 1.0, 0.0)), term(0.3, None, (QUAD, 1.0, 0.0)),
                term(0.3, None, None, (QUAD, 1.0, 0.0)))
    sigma = sst(term(1.0), term(1.0, (LIN, 1.0, 0.0), (LIN, 1.0, 0.0)))
    phi = sst(term(1.0, (LIN, 1.0, 0.0), (SIN, 2 * PI, 0.0)),
              term(1.0 / (2 * PI), None, None, (SIN, 2 * PI, 0.0)),
              term(0.5, None, None, (LIN, 1.0, 0.0)))
    return problem(3, box([0, 0, 0], [1, 1, 1]), alpha, sigma, manufactured(), u, phi=phi, um=u)


def cube3d_literal_problem():
    """The 3D cube workload with its literal drift omega = (sin 2 pi y, cos 2 pi z, 0.5)
    (non-zero curl: not alpha times a gradient), u, alpha, sigma as in cube3d_problem;
    f from eq. 1.  Needs the extra-drift walk (the paper has no exact estimator for it)."""
    u = sst(term(1.0, (EXP, 0.5, 0.0), (SIN, PI, 0.0), (COS, PI, 0.0)))
    alpha = sst(term(1.0), term(0.3, (QUAD, 1.0, 0.0)), term(0.3, None, (QUAD, 1.0, 0.0)),
                term(0.3, None, None, (QUAD, 1.0, 0.0)))
    sigma = sst(term(1.0), term(1.0, (LIN, 1.0, 0.0), (LIN, 1.0, 0.0)))
    omega = [sst(term(1.0, None, (SIN, 2 * PI, 0.0))), sst(term(1.0, None, None, (COS, 2 * PI, 0.0))),
             const(0.5)]
    # |omega| <= (1 + 1 + 0.25)^(1/2) = 1.5 and alpha >= 1 on the cube: |omega / alpha| <= 1.5
    return problem(3, box([0, 0, 0], [1, 1, 1]), alpha, sigma, manufactured(), u, um=u, omega=omega,
                   drift_bound=1.5)


def cube3d_exact(x, y, z):
    return np.exp(0.5 * x) * np.sin(np.pi * y) * np.cos(np.pi * z)


def cube3d_exact_grad(x, y, z):
    """grad u of cube3d_exact, shape [3, ...]."""
    e = np.exp(0.5 * x)
    return np.array([0.5 * e * np.sin(np.pi * y) * np.cos(np.pi * z),
                     np.pi * e * np.cos(np.pi * y) * np.cos(np.pi * z),
                     -np.pi * e * np.sin(np.pi * y) * np.sin(np.pi * z)])


CUBE3D = {"name": "cube3d_drift_manufactured", "eps": 1e-4, "grid": 64, "walks": 1024,
          "seed": 0}


# ---------------------------------------------------------------------------
# Closed-form test families (Sec. 2.3-2.4): harmonic g (Kakutani), constant
# screening with a known solution.
# ---------------------------------------------------------------------------
def laplace_disk_problem():
    """Delta u = 0 on the unit disk, u = x^2 - y^2."""
    u = sst(term(1.0, (QUAD, 1.0, 0.0)), term(-1.0, None, (QUAD, 1.0, 0.0)))
    return problem(2, ball([0, 0], 1.0), const(1.0), zero(), zero(), u, um=u)


def laplace_disk_exact(x, y):
    return x * x - y * y


def laplace_disk_exact_grad(x, y):
    return np.array([2.0 * x, -2.0 * y])


def laplace_ball_problem():
    """Delta u = 0 on the unit ball, u = x y z + x^2 - z^2."""
    u = sst(term(1.0, (LIN, 1.0, 0.0), (LIN, 1.0, 0.0), (LIN, 1.0, 0.0)),
            term(1.0, (QUAD, 1.0, 0.0)), term(-1.0, None, None, (QUAD, 1.0, 0.0)))
    return problem(3, ball([0, 0, 0], 1.0), const(1.0), zero(), zero(), u, um=u)


def laplace_ball_exact(x, y, z):
    return x * y * z + x * x - z * z


def laplace_ball_exact_grad(x, y, z):
    return np.array([y * z + 2.0 * x, x * z, x * y - 2.0 * z])


def screened_square_problem(sig=4.0):
    """Delta u - sigma u = -f on the unit square with u = sin(x) sin(y), f = (2 + sigma) u."""
    u = sst(term(1.0, (SIN, 1.0, 0.0), (SIN, 1.0, 0.0)))
    return problem(2, box([0, 0], [1, 1]), const(1.0), const(sig), manufactured(), u, um=u)


def screened_square_exact(x, y):
    return np.sin(x) * np.sin(y)


def screened_ball_problem(sig=9.0):
    """Delta u - sigma u = 0 on the unit ball with u = cosh(sqrt(sigma) x)."""
    s = math.sqrt(sig)
    u = sst(term(1.0, (COSH, s, 0.0)))
    return problem(3, ball([0, 0, 0], 1.0), const(1.0), const(sig), manufactured(), u, um=u)


def screened_ball_exact(sig, x, y, z):
    return np.cosh(np.sqrt(sig) * x)


def screened_ball_exact_grad(sig, x, y, z):
    s = np.sqrt(sig)
    return np.array([s * np.sinh(s * x), 0.0 * y, 0.0 * z])


# ---------------------------------------------------------------------------
# evaluation points (SoA float32 [dim][npts])
# ---------------------------------------------------------------------------
def cell_centres(dim, n, lo=0.0, hi=1.0):
    """Cell centres of an n^dim grid on [lo, hi]^dim; x varies fastest (C-contiguous SoA)."""
    c = (np.arange(n, dtype=np.float64) + 0.5) / n * (hi - lo) + lo
    mesh = np.meshgrid(*([c] * dim), indexing="ij")
    # x fastest: reverse the axis order of the flattened index
    pts = np.stack([m.transpose(tuple(range(dim))[::-1]).reshape(-1) for m in mesh])
    return pts.astype(np.float32)


def seeded_subset(npts, m, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(npts, size=min(m, npts), replace=False))


def uniform_in_ball(dim, n, centre, radius, seed, margin=0.0):
    rng = np.random.default_rng(seed)
    out = []
    while sum(len(o) for o in out) < n:
        x = rng.uniform(-1.0, 1.0, size=(4 * n, dim))
        r = np.linalg.norm(x, axis=1)
        out.append(x[r < 1.0 - margin])
    x = np.concatenate(out)[:n] * radius + np.asarray(centre[:dim])
    return np.ascontiguousarray(x.T.astype(np.float32))


def uniform_in_box(dim, n, lo, hi, seed):
    """n uniform points in the box [lo, hi] (scalars or per-axis bounds), SoA float32."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo, hi, size=(n, dim))
    return np.ascontiguousarray(x.T.astype(np.float32))


# ---------------------------------------------------------------------------
# seeded value-noise grids: a lattice of uniform random values every `cell`
# nodes, interpolated with the quintic fade 6t^5 - 15t^4 + 10t^3 (C^2) onto the
# node grid and mapped affinely to [vmin, vmax]
# ---------------------------------------------------------------------------
def value_noise_grid(dim, res, vmin, vmax, seed, cell=8):
    rng = np.random.default_rng(seed)
    nl = (res - 1) // cell + 2
    lattice = rng.uniform(0.0, 1.0, size=(nl,) * dim)
    s = np.arange(res, dtype=np.float64) / cell
    i0 = np.minimum(np.floor(s).astype(np.int64), nl - 2)
    t = s - i0
    w = t * t * t * (t * (t * 6.0 - 15.0) + 10.0)
    out = np.zeros((res,) * dim)
    for corner in range(1 << dim):
        idx = []
        wt = np.ones((res,) * dim)
        for d in range(dim):
            o = (corner >> d) & 1
            shape = [1] * dim
            shape[dim - 1 - d] = res          # axis d is the (dim-1-d)-th array axis (x fastest)
            wd = (w if o else 1.0 - w).reshape(shape)
            wt = wt * wd
            idx.append((i0 + o).reshape(shape))
        # lattice indexed [z][y][x]
        out += wt * lattice[tuple(idx[::-1])]
    return (vmin + (vmax - vmin) * out).astype(np.float32)


def grid_field(kind, data, lo, hi):
    res = list(data.shape[::-1])
    return {"kind": kind, "res": res, "lo": list(lo), "hi": list(hi), "data": data}


def noise_cube_problem(res=33, seed=11):
    """Unit cube with noise coefficients: alpha in [0.5, 2] (cubic B-spline),
    sigma in [0, 20] and f in [-1, 1] (multilinear), g = x y + z."""
    lo, hi = [0.0, 0.0, 0.0], [1.0, 1.0, 1.0]
    a = value_noise_grid(3, res, 0.5, 2.0, seed, cell=8)
    s = value_noise_grid(3, res, 0.0, 20.0, seed + 1, cell=8)
    f = value_noise_grid(3, res, -1.0, 1.0, seed + 2, cell=8)
    g = sst(term(1.0, (LIN, 1.0, 0.0), (LIN, 1.0, 0.0)), term(1.0, None, None, (LIN, 1.0, 0.0)))
    return problem(3, box(lo, hi), grid_field("grid_bspline", a, lo, hi),
                   grid_field("grid_linear", s, lo, hi), grid_field("grid_linear", f, lo, hi), g)


def noise_annulus_problem(seed=21):
    """2D annulus with a B-spline noise alpha, a noise drift potential and a screening field."""
    lo, hi = [-1.2, -1.2], [1.2, 1.2]
    a = value_noise_grid(2, 49, 0.5, 2.0, seed, cell=8)
    ph = value_noise_grid(2, 49, -0.5, 0.5, seed + 1, cell=8)
    s = value_noise_grid(2, 49, 0.0, 10.0, seed + 2, cell=8)
    g = sst(term(1.0, (COS, PI, 0.0), (LIN, 1.0, 0.0)))
    f = sst(term(1.0, (SIN, 2.0, 0.0), (COS, 3.0, 0.0)))
    return problem(2, annulus([0.0, 0.0], 0.35, 1.1), grid_field("grid_bspline", a, lo, hi),
                   grid_field("grid_linear", s, lo, hi), f, g,
                   phi=grid_field("grid_bspline", ph, lo, hi))


def rounded_box_problem():
    """2D rounded box, alpha = 1 + 0.3 sin(2x) sin(3y), sigma = 3, manufactured u = cos(x) e^{0.5 y}."""
    u = sst(term(1.0, (COS, 1.0, 0.0), (EXP, 0.5, 0.0)))
    alpha = sst(term(1.0), term(0.3, (SIN, 2.0, 0.0), (SIN, 3.0, 0.0)))
    return problem(2, rounded_box([0.1, -0.2], [1.0, 0.7], 0.3), alpha, const(3.0), manufactured(), u, um=u)


def rounded_box_exact(x, y):
    return np.cos(x) * np.exp(0.5 * y)


# ---------------------------------------------------------------------------
# Mesh workload: a displaced icosphere.  An icosahedron subdivided `level` times
# (20 * 4^level triangles; level 7 = 327,680, the nearest icosphere to 2^18),
# vertices on the unit sphere displaced radially to r = 1 + amp * n(v), with n a
# seeded 3D value noise in [-1, 1] (lattice spacing 0.25, quintic fade).  The
# surface stays star-shaped about the origin, closed and consistently oriented.
# ---------------------------------------------------------------------------
def icosphere(level):
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4], [11, 10, 2],
                  [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9], [4, 9, 5],
                  [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    for _ in range(level):
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
        key = np.sort(e, axis=1)
        uniq, inv = np.unique(key[:, 0] * len(v) + key[:, 1], return_inverse=True)
        a, b = uniq // len(v), uniq % len(v)
        mid = v[a] + v[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        m = inv.reshape(3, -1).T + len(v)  # midpoints of edges (01, 12, 20) per face
        v = np.concatenate([v, mid])
        f = np.concatenate([np.stack([f[:, 0], m[:, 0], m[:, 2]], 1), np.stack([f[:, 1], m[:, 1], m[:, 0]], 1),
                            np.stack([f[:, 2], m[:, 2], m[:, 1]], 1), m])
    return v, f


def value_noise_3d(x, seed, spacing=0.25, extent=2.0):
    """Seeded value noise in [-1, 1] at points x (n x 3), lattice spacing `spacing` on [-extent, extent]^3."""
    rng = np.random.default_rng(seed)
    n = int(round(2 * extent / spacing)) + 2
    lattice = rng.uniform(-1.0, 1.0, size=(n, n, n))
    s = (np.asarray(x, dtype=np.float64) + extent) / spacing
    i0 = np.clip(np.floor(s).astype(np.int64), 0, n - 2)
    t = s - i0
    w = t * t * t * (t * (t * 6.0 - 15.0) + 10.0)
    out = np.zeros(len(s))
    for c in range(8):
        o = [(c >> d) & 1 for d in range(3)]
        wt = np.ones(len(s))
        for d in range(3):
            wt *= w[:, d] if o[d] else 1.0 - w[:, d]
        out += wt * lattice[i0[:, 0] + o[0], i0[:, 1] + o[1], i0[:, 2] + o[2]]
    return out


def displaced_icosphere(level=7, amplitude=0.1, seed=3):
    """Vertices (float32 n x 3) and triangles (int32 m x 3) of the displaced icosphere."""
    v, f = icosphere(level)
    r = 1.0 + amplitude * value_noise_3d(v, seed)
    return (v * r[:, None]).astype(np.float32), f.astype(np.int32)


def mesh_domain(verts, tris, grid_res=0, tol=0.0):
    """Closed triangle mesh; grid_res > 0 adds a grid_res^3 distance grid (conservative radii);
    tol > 0 lets distance queries stop at a certified radius >= (1 - tol) x the distance."""
    return {"kind": "mesh", "p": [0.0] * 16, "verts": verts, "tris": tris, "grid_res": int(grid_res),
            "tol": float(tol)}


def mesh_noise_problem(level=7, grid_res=128, seed=3, dist_grid=0, tol=0.0):
    """Displaced icosphere boundary; alpha in [0.5, 2] (cubic B-spline), sigma in [0, 20] and
    f in [-1, 1] (multilinear) from seeded 128^3 value-noise grids over the mesh box plus 5%;
    g = x y + z."""
    verts, tris = displaced_icosphere(level, 0.1, seed)
    lo = verts.min(axis=0).astype(np.float64)
    hi = verts.max(axis=0).astype(np.float64)
    pad = 0.05 * (hi - lo)
    lo, hi = list(lo - pad), list(hi + pad)
    a = value_noise_grid(3, grid_res, 0.5, 2.0, seed + 1, cell=8)
    s = value_noise_grid(3, grid_res, 0.0, 20.0, seed + 2, cell=8)
    f = value_noise_grid(3, grid_res, -1.0, 1.0, seed + 3, cell=8)
    g = sst(term(1.0, (LIN, 1.0, 0.0), (LIN, 1.0, 0.0)), term(1.0, None, None, (LIN, 1.0, 0.0)))
    return problem(3, mesh_domain(verts, tris, dist_grid, tol), grid_field("grid_bspline", a, lo, hi),
                   grid_field("grid_linear", s, lo, hi), grid_field("grid_linear", f, lo, hi), g)


def mesh_interior_points(n, seed, radius=0.88):
    """Uniform points in the ball of radius 0.88: inside the displaced icosphere, whose
    vertices lie at r >= 0.9 and whose flat triangles dip below that by < 1e-4."""
    return uniform_in_ball(3, n, [0.0, 0.0, 0.0], radius, seed)


def mesh_manufactured_problem(level=5, amplitude=0.1, seed=3, dist_grid=0, tol=0.0):
    """The 3D manufactured problem (u, alpha, sigma, drift of the cube workload) on the
    displaced-icosphere domain: u is exact on any domain, so the mesh walk has an exact answer."""
    verts, tris = displaced_icosphere(level, amplitude, seed)
    p = cube3d_problem()
    p["domain"] = mesh_domain(verts, tris, dist_grid, tol)
    return p


# ---------------------------------------------------------------------------
# Inverse problem: recover a 32^3 multilinear sigma grid on the unit cube from
# the solution at seeded sensors.  alpha: 16^3 cubic B-spline noise in [0.5, 2]
# (seed 2, fixed); hidden sigma: 32^3 noise in [0, 10] (seed 1); f = 1;
# g = 1 + x y + z; sensors uniform in [0.05, 0.95]^3.
# ---------------------------------------------------------------------------
def inverse_alpha_grid(seed=2):
    return value_noise_grid(3, 16, 0.5, 2.0, seed, cell=8)


def inverse_sigma_grid(seed=1):
    return value_noise_grid(3, 32, 0.0, 10.0, seed, cell=8)


def inverse_problem(sigma_grid, alpha_grid=None):
    lo, hi = [0.0, 0.0, 0.0], [1.0, 1.0, 1.0]
    alpha = inverse_alpha_grid() if alpha_grid is None else alpha_grid
    g = sst(term(1.0), term(1.0, (LIN, 1.0, 0.0), (LIN, 1.0, 0.0)), term(1.0, None, None, (LIN, 1.0, 0.0)))
    return problem(3, box(lo, hi), grid_field("grid_bspline", alpha, lo, hi),
                   grid_field("grid_linear", sigma_grid, lo, hi), const(1.0), g)


def inverse_sensors(n=4096, seed=4):
    return uniform_in_box(3, n, 0.05, 0.95, seed)


# ---------------------------------------------------------------------------
# Batched uneven solves: independent 2D problems (disks, annuli, rounded boxes,
# seeded sizes 0.5 - 2), each with its own 64^2 noise grids: alpha in [0.5, 2]
# (B-spline), sigma in [0, 10] and f in [-1, 1] (multilinear), a drift potential
# Phi (B-spline) scaled so |omega| = |alpha grad Phi| <= 2 on its grid; g =
# cos(pi x) y.  Points per problem log-uniform in [16, 4096], walks per point
# log-uniform in [64, 1024].  The drift is conservative by construction (App. A).
# ---------------------------------------------------------------------------
def _inside_2d(dom, x, y, margin=0.0):
    p = dom["p"]
    if dom["kind"] == "ball":
        return np.hypot(x - p[0], y - p[1]) < p[3] - margin
    if dom["kind"] == "annulus":
        r = np.hypot(x - p[0], y - p[1])
        return (r > p[3] + margin) & (r < p[4] - margin)
    # rounded box: inside when the distance to the inner box is below the corner radius
    qx = np.abs(x - p[0]) - (p[3] - p[6])
    qy = np.abs(y - p[1]) - (p[4] - p[6])
    out = np.hypot(np.maximum(qx, 0), np.maximum(qy, 0)) + np.minimum(np.maximum(qx, qy), 0)
    return out < p[6] - margin


def batch_problems(nprob, seed=7, grid=64, max_points=4096, min_points=16, min_walks=64, max_walks=1024):
    """(problems, points SoA float32 [2][N], offsets [nprob+1], walks int32 [N])."""
    rng = np.random.default_rng(seed)
    probs, pts, offs, walks = [], [], [0], []
    g = sst(term(1.0, (COS, PI, 0.0), (LIN, 1.0, 0.0)))
    for i in range(nprob):
        kind = int(rng.integers(0, 3))
        c = rng.uniform(-1.0, 1.0, size=2)
        if kind == 0:
            r = rng.uniform(0.5, 2.0)
            dom = ball(c, r)
            half = np.array([r, r])
        elif kind == 1:
            r = rng.uniform(0.5, 2.0)
            dom = annulus(c, r * rng.uniform(0.3, 0.7), r)
            half = np.array([r, r])
        else:
            half = rng.uniform(0.5, 2.0, size=2)
            dom = rounded_box(c, half, rng.uniform(0.1, 0.4) * half.min())
        lo, hi = list(c - half), list(c + half)
        s = int(rng.integers(0, 2 ** 31))
        a = value_noise_grid(2, grid, 0.5, 2.0, s, cell=8)
        sg = value_noise_grid(2, grid, 0.0, 10.0, s + 1, cell=8)
        f = value_noise_grid(2, grid, -1.0, 1.0, s + 2, cell=8)
        ph = value_noise_grid(2, grid, -1.0, 1.0, s + 3, cell=8).astype(np.float64)
        h = (np.array(hi) - np.array(lo)) / (grid - 1)
        gy, gx = np.gradient(ph, h[1], h[0])
        wmax = np.max(a * np.hypot(gx, gy))
        ph = (ph * (2.0 / wmax)).astype(np.float32)
        probs.append(problem(2, dom, grid_field("grid_bspline", a, lo, hi), grid_field("grid_linear", sg, lo, hi),
                             grid_field("grid_linear", f, lo, hi), g, phi=grid_field("grid_bspline", ph, lo, hi)))
        n = int(round(np.exp(rng.uniform(np.log(min_points), np.log(max_points)))))
        got = []
        while sum(len(q) for q in got) < n:
            x = rng.uniform(lo[0], hi[0], size=4 * n)
            y = rng.uniform(lo[1], hi[1], size=4 * n)
            m = _inside_2d(dom, x, y, margin=1e-3)
            got.append(np.stack([x[m], y[m]], 1))
        q = np.concatenate(got)[:n]
        pts.append(q)
        offs.append(offs[-1] + n)
        walks.append(np.round(np.exp(rng.uniform(np.log(min_walks), np.log(max_walks), size=n))).astype(np.int32))
    P = np.ascontiguousarray(np.concatenate(pts).T.astype(np.float32))
    return probs, P, np.array(offs, dtype=np.int64), np.concatenate(walks)


def fd_square_problem():
    """A unit-square problem with closed-form coefficients and no closed-form solution:
    alpha = 1 + 0.5 sin(2 pi x) cos(2 pi y), omega = alpha grad(Phi) with Phi = 0.5 x y,
    sigma = 2 + sin(3x + y), f = 1 + x, g = x^2 + y (reference: a fine finite-difference
    solve)."""
    alpha = sst(term(1.0), term(0.5, (SIN, 2 * PI, 0.0), (COS, 2 * PI, 0.0)))
    phi = sst(term(0.5, (LIN, 1.0, 0.0), (LIN, 1.0, 0.0)))
    sigma = sst(term(2.0), term(1.0, (SIN, 3.0, 0.0), (COS, 1.0, 0.0)),
                term(1.0, (COS, 3.0, 0.0), (SIN, 1.0, 0.0)))
    f = sst(term(1.0), term(1.0, (LIN, 1.0, 0.0)))
    g = sst(term(1.0, (QUAD, 1.0, 0.0)), term(1.0, None, (LIN, 1.0, 0.0)))
    return problem(2, box([0, 0], [1, 1]), alpha, sigma, f, g, phi=phi)


def fd_square_coefficients():
    """The same coefficients as numpy functions of (x, y): alpha, grad Phi, sigma, f, g."""
    return {
        "alpha": lambda x, y: 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y),
        "grad_phi": lambda x, y: (0.5 * y, 0.5 * x),
        "sigma": lambda x, y: 2.0 + np.sin(3.0 * x + y),
        "f": lambda x, y: 1.0 + x,
        "g": lambda x, y: x * x + y,
    }


def hifreq_alpha_problem(freq=6.0, amp=0.8):
    """div(alpha grad u) = -f on the unit square with a high-frequency diffusion
    coefficient alpha = 1 + amp sin(freq pi x) sin(freq pi y), u = sin(pi x) sinh(y) / sinh(1) + 1
    (the setting of the paper's weight-window experiment, Sec. 6)."""
    u = sst(term(1.0), term(1.0 / math.sinh(1.0), (SIN, PI, 0.0), (SINH, 1.0, 0.0)))
    alpha = sst(term(1.0), term(amp, (SIN, freq * PI, 0.0), (SIN, freq * PI, 0.0)))
    return problem(2, box([0, 0], [1, 1]), alpha, zero(), manufactured(), u, um=u)


def hifreq_alpha_exact(x, y):
    return np.sin(np.pi * x) * np.sinh(y) / np.sinh(1.0) + 1.0


def hifreq_alpha_exact_grad(x, y):
    k = 1.0 / np.sinh(1.0)
    return np.array([np.pi * np.cos(np.pi * x) * np.sinh(y) * k, np.sin(np.pi * x) * np.cosh(y) * k])



# ---------------------------------------------------------------------------
# Signed-distance CSG scenes (Sec. 7.2: domains edited as a list of SDF CSG
# operations).  Harmonic boundary data make the exact solution the data itself.
# ---------------------------------------------------------------------------
def csg_scene_2d():
    """Union of two disks minus a smaller disk and a box notch."""
    return csg([-1.2, -1.0], [1.6, 1.0],
               ("sphere", "union", [0.0, 0.0, 0.0, 0.9]),
               ("sphere", "union", [0.8, 0.1, 0.0, 0.7]),
               ("sphere", "subtract", [0.25, -0.15, 0.0, 0.3]),
               ("box", "subtract", [-0.6, 0.7, 0.0, 0.25, 0.35, 0.0, 0.05]))


def csg_scene_3d():
    """A rounded box with a spherical cavity, a capsule added through it and a half-space cut."""
    return csg([-1.3, -1.3, -1.3], [1.3, 1.3, 1.3],
               ("box", "union", [0.0, 0.0, 0.0, 0.9, 0.7, 0.6, 0.15]),
               ("capsule", "union", [-1.1, 0.0, 0.0, 1.1, 0.0, 0.0, 0.3]),
               ("sphere", "subtract", [0.3, 0.2, 0.1, 0.35]),
               ("torus", "subtract", [0.0, 0.0, 0.6, 0.45, 0.12]),
               ("halfspace", "intersect", [0.0, -0.5, 0.0, 0.0, -1.0, 0.0]))


def csg_laplace_problem(dim):
    """Laplace's equation on a CSG scene with harmonic g (u = g): 2D x^2 - y^2 + x, 3D xyz + x^2 - z^2."""
    if dim == 2:
        u = sst(term(1.0, (QUAD, 1.0, 0.0)), term(-1.0, None, (QUAD, 1.0, 0.0)), term(1.0, (LIN, 1.0, 0.0)))
        return problem(2, csg_scene_2d(), const(1.0), zero(), zero(), u, um=u)
    u = sst(term(1.0, (LIN, 1.0, 0.0), (LIN, 1.0, 0.0), (LIN, 1.0, 0.0)),
            term(1.0, (QUAD, 1.0, 0.0)), term(-1.0, None, None, (QUAD, 1.0, 0.0)))
    return problem(3, csg_scene_3d(), const(1.0), zero(), zero(), u, um=u)


def csg_laplace_exact(dim, x):
    if dim == 2:
        return x[0] ** 2 - x[1] ** 2 + x[0]
    return x[0] * x[1] * x[2] + x[0] ** 2 - x[2] ** 2


def csg_variable_problem():
    """The 3D CSG scene with variable coefficients and a manufactured solution."""
    u = sst(term(1.0, (EXP, 0.5, 0.0), (SIN, PI, 0.0), (COS, PI, 0.0)))
    alpha = sst(term(1.0), term(0.3, (QUAD, 1.0, 0.0)), term(0.3, None, (QUAD, 1.0, 0.0)))
    sigma = sst(term(1.0), term(1.0, (LIN, 1.0, 0.0), (LIN, 1.0, 0.0)))
    return problem(3, csg_scene_3d(), alpha, sigma, manufactured(), u, um=u)
