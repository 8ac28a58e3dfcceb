"""Second-order finite-difference reference solve of eq. 1 on the unit square.

div(alpha grad u) + omega . grad u - sigma u = -f with omega = alpha grad Phi and
u = g on the boundary, discretised on an N x N cell grid (nodes i h, h = 1/N):
the flux form with alpha at the half nodes for the diffusion term, central
differences for the drift, and the boundary values moved to the right-hand
side.  Solved with a sparse direct solver.  Independent of the walk code: it
uses only the closed-form coefficient functions.
"""
import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla


def fd_solve_square(c, n):
    """Nodal solution u[(n+1), (n+1)] (index [i, j] at x = i h, y = j h)."""
    h = 1.0 / n
    xs = np.arange(n + 1) * h
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    u = np.zeros((n + 1, n + 1))
    u[0, :], u[n, :] = c["g"](X[0, :], Y[0, :]), c["g"](X[n, :], Y[n, :])
    u[:, 0], u[:, n] = c["g"](X[:, 0], Y[:, 0]), c["g"](X[:, n], Y[:, n])
    m = n - 1
    idx = -np.ones((n + 1, n + 1), dtype=np.int64)
    idx[1:n, 1:n] = np.arange(m * m).reshape(m, m)
    I, J = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="ij")
    I, J = I.ravel(), J.ravel()
    x, y = I * h, J * h
    ae = c["alpha"](x + 0.5 * h, y)
    aw = c["alpha"](x - 0.5 * h, y)
    an = c["alpha"](x, y + 0.5 * h)
    as_ = c["alpha"](x, y - 0.5 * h)
    a0 = c["alpha"](x, y)
    px, py = c["grad_phi"](x, y)
    wx, wy = a0 * px, a0 * py
    sig = c["sigma"](x, y)
    rows, cols, vals = [], [], []
    rhs = -c["f"](x, y) * h * h
    row = idx[I, J]
    diag = -(ae + aw + an + as_) - sig * h * h
    rows.append(row)
    cols.append(row)
    vals.append(diag)
    for di, dj, coef in ((1, 0, ae + 0.5 * h * wx), (-1, 0, aw - 0.5 * h * wx),
                         (0, 1, an + 0.5 * h * wy), (0, -1, as_ - 0.5 * h * wy)):
        nb = idx[I + di, J + dj]
        inner = nb >= 0
        rows.append(row[inner])
        cols.append(nb[inner])
        vals.append(coef[inner])
        rhs[~inner] -= coef[~inner] * u[(I + di)[~inner], (J + dj)[~inner]]
    A = sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(m * m, m * m))
    u[1:n, 1:n] = spla.spsolve(A, rhs).reshape(m, m)
    return u


def fd_reference_at(c, pts, n=512):
    """u at points that lie on the nodes of the n-grid (pts [2, npts] multiples of 1/n)."""
    u = fd_solve_square(c, n)
    ij = np.rint(np.asarray(pts, dtype=np.float64) * n).astype(np.int64)
    assert np.allclose(ij / n, pts, atol=1e-7), "points must be grid nodes"
    return u[ij[0], ij[1]]


# ---------------------------------------------------------------------------
# 3D: div(alpha grad u) - sigma u = -f on the unit cube, u = g on the boundary,
# with alpha a clamped cubic B-spline grid (node values as control points) and
# sigma a multilinear grid, both spanning [0, 1]^3 with array index [z, y, x].
# The discrete adjoint gives the gradient of a linear functional of u with
# respect to the sigma grid (the reference for the path-replay adjoint).
# ---------------------------------------------------------------------------
def _bspline_w(t):
    u = 1.0 - t
    return np.stack([u ** 3 / 6.0, (3 * t ** 3 - 6 * t ** 2 + 4) / 6.0, (-3 * t ** 3 + 3 * t ** 2 + 3 * t + 1) / 6.0,
                     t ** 3 / 6.0])


def bspline3(grid, x, y, z):
    """Clamped cubic B-spline with control points at the grid nodes, nodes at i / (res - 1)."""
    res = grid.shape[0]
    out = np.zeros(np.broadcast(x, y, z).shape)
    idx, wts = [], []
    for c in (x, y, z):
        s = np.asarray(c, dtype=np.float64) * (res - 1)
        fs = np.floor(s)
        idx.append(fs.astype(np.int64) - 1)
        wts.append(_bspline_w(s - fs))
    for a in range(4):
        ia = np.clip(idx[0] + a, 0, res - 1)
        for b in range(4):
            ib = np.clip(idx[1] + b, 0, res - 1)
            for c in range(4):
                ic = np.clip(idx[2] + c, 0, res - 1)
                out += wts[0][a] * wts[1][b] * wts[2][c] * grid[ic, ib, ia]
    return out


def multilinear_weights(res, x, y, z):
    """(node index arrays, weights) of the multilinear interpolation at the points."""
    i0, t = [], []
    for c in (x, y, z):
        s = np.clip(np.asarray(c, dtype=np.float64) * (res - 1), 0, res - 1)
        i = np.minimum(np.floor(s).astype(np.int64), res - 2)
        i0.append(i)
        t.append(s - i)
    nodes, wts = [], []
    for corner in range(8):
        o = [(corner >> d) & 1 for d in range(3)]
        w = np.ones_like(t[0])
        for d in range(3):
            w = w * (t[d] if o[d] else 1.0 - t[d])
        nodes.append((i0[0] + o[0]) + res * ((i0[1] + o[1]) + res * (i0[2] + o[2])))
        wts.append(w)
    return nodes, wts


def fd_cube_operator(alpha_grid, sigma_grid, f, g, n):
    """Matrix A, right-hand side b (A u = b on interior nodes) and helpers on an n-interval grid."""
    h = 1.0 / n
    m = n - 1
    ii = np.arange(1, n)
    Z, Y, X = np.meshgrid(ii, ii, ii, indexing="ij")
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    x, y, z = X * h, Y * h, Z * h
    row = (X - 1) + m * ((Y - 1) + m * (Z - 1))
    res_s = sigma_grid.shape[0]
    nodes, wts = multilinear_weights(res_s, x, y, z)
    sflat = sigma_grid.reshape(-1).astype(np.float64)
    sig = sum(w * sflat[nd] for nd, w in zip(nodes, wts))
    rows, cols, vals = [row], [row], [sig * h * h]
    b = f(x, y, z) * h * h
    diag = sig * h * h
    for d, (dx, dy, dz) in enumerate(((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))):
        a = bspline3(alpha_grid, x + 0.5 * dx * h, y + 0.5 * dy * h, z + 0.5 * dz * h)
        diag = diag + a
        Xn, Yn, Zn = X + dx, Y + dy, Z + dz
        inner = (Xn >= 1) & (Xn <= m) & (Yn >= 1) & (Yn <= m) & (Zn >= 1) & (Zn <= m)
        nb = (Xn - 1) + m * ((Yn - 1) + m * (Zn - 1))
        rows.append(row[inner])
        cols.append(nb[inner])
        vals.append(-a[inner])
        b[~inner] += a[~inner] * g(Xn[~inner] * h, Yn[~inner] * h, Zn[~inner] * h)
    vals[0] = diag
    A = sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(m ** 3, m ** 3))
    return A, b, (x, y, z, row, nodes, wts)


def fd_cube_sensor_matrix(n, pts, g):
    """Trilinear interpolation of the nodal solution at sensor points: u(pts) = S u_int + c."""
    h = 1.0 / n
    m = n - 1
    rows, cols, vals = [], [], []
    c = np.zeros(pts.shape[1])
    s = pts / h
    i0 = np.minimum(np.floor(s).astype(np.int64), n - 1)
    t = s - i0
    for corner in range(8):
        o = np.array([(corner >> d) & 1 for d in range(3)])[:, None]
        w = np.prod(np.where(o == 1, t, 1.0 - t), axis=0)
        idx = i0 + o
        interior = np.all((idx >= 1) & (idx <= m), axis=0)
        p_in = np.nonzero(interior)[0]
        rows.append(p_in)
        cols.append((idx[0, p_in] - 1) + m * ((idx[1, p_in] - 1) + m * (idx[2, p_in] - 1)))
        vals.append(w[p_in])
        p_b = np.nonzero(~interior)[0]
        c[p_b] += w[p_b] * g(idx[0, p_b] * h, idx[1, p_b] * h, idx[2, p_b] * h)
    S = sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(pts.shape[1], m ** 3))
    return S, c


def fd_cube_sigma_gradient(alpha_grid, sigma_grid, f, g, n, pts, w):
    """(u at the sensors, d(sum_p w_p u(x_p)) / d sigma grid nodes) of the finite-difference solution."""
    A, b, (x, y, z, row, nodes, wts) = fd_cube_operator(alpha_grid, sigma_grid, f, g, n)
    # A is symmetric positive definite (flux form, sigma >= 0): conjugate gradients with Jacobi
    M = sps.diags(1.0 / A.diagonal())
    u, info = spla.cg(A, b, rtol=1e-12, atol=0.0, maxiter=20000, M=M)
    assert info == 0
    S, c = fd_cube_sensor_matrix(n, pts, g)
    lam, info = spla.cg(A, S.T @ w, rtol=1e-12, atol=0.0, maxiter=20000, M=M)
    assert info == 0
    h = 1.0 / n
    grad = np.zeros(sigma_grid.size)
    for nd, wt in zip(nodes, wts):
        np.add.at(grad, nd, -lam[row] * wt * u[row] * h * h)
    return S @ u + c, grad
