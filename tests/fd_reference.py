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
