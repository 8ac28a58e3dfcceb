"""GPU parity of the CUDA walk kernels (through the C interface) with the FP64 oracle.

* FP64 replay: the same Philox streams must give the oracle's walk, per walk,
  to 1e-9 (relative to max(1, |u|)) on >= 99% of walks, with equal step counts.
* FP32 production path: per-point agreement within 4 combined standard errors
  at matched walk counts (read for many points as in tests/stats_util.py).
* Accuracy: normalised RMS error <= 1e-2 against the manufactured solution at
  2^16 walks per point.
* The full-size 3D workload in the benchmark's launch configuration, checked on
  sampled points against the oracle.
* Edge cases: empty and ragged inputs, per-point walk counts with zeros, walk-id
  continuation, points in the epsilon shell, invalid arguments.
"""
import numpy as np
import pytest

import workloads as W
from tests.stats_util import combined_z, four_se_rule, normalised_rms

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wos():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_13240_gb300 import build as B
    B.build_lib()
    import paper_2201_13240_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(wos):
    return wos.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


REPLAY_CASES = {
    "square2d": (W.square2d_problem, lambda: W.cell_centres(2, 32)[:, W.seeded_subset(1024, 48, 1)], 1e-3),
    "cube3d": (W.cube3d_problem, lambda: W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 48, 2)], 1e-4),
    "laplace_disk": (W.laplace_disk_problem, lambda: W.uniform_in_ball(2, 48, [0, 0], 1.0, 3, 0.02), 1e-4),
    "screened_ball": (W.screened_ball_problem, lambda: W.uniform_in_ball(3, 48, [0, 0, 0], 1.0, 4, 0.02), 1e-4),
    "rounded_box": (W.rounded_box_problem,
                    lambda: W.uniform_in_box(2, 48, [-0.6, -0.6], [0.8, 0.2], 5), 1e-3),
    "noise_annulus": (W.noise_annulus_problem,
                      lambda: np.array([[0.5, -0.6, 0.0, 0.7, -0.4, 0.2], [0.2, 0.3, -0.8, -0.5, -0.5, 0.9]],
                                       dtype=np.float32), 1e-3),
    "noise_cube": (W.noise_cube_problem, lambda: W.uniform_in_box(3, 24, 0.1, 0.9, 6), 1e-3),
    "mesh": (lambda: W.mesh_manufactured_problem(level=5), lambda: W.mesh_interior_points(32, 7), 1e-4),
    "mesh_grid": (lambda: W.mesh_manufactured_problem(level=5, dist_grid=48), lambda: W.mesh_interior_points(32, 7),
                  1e-4),
}


@pytest.mark.parametrize("name", list(REPLAY_CASES))
def test_fp64_replay_matches_oracle_per_walk(orc, ctx, name):
    mk, ptsf, eps = REPLAY_CASES[name]
    desc = mk()
    pts = ptsf()
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc, 64 if desc["dim"] == 3 else 128)[0]
    wpp = 16
    uh, st, stats = ctx.walk_estimates(prob, dev(pts), wpp, eps, sb, seed=7, precision="fp64")
    uo, so = orc.walks(desc, pts, wpp, seed=7, eps=eps, sigma_bar=sb)
    uh = uh.cpu().numpy()
    st = st.cpu().numpy()
    ok = np.abs(uh - uo) <= 1e-9 * np.maximum(1.0, np.abs(uo))
    assert ok.mean() >= 0.99, (name, ok.mean(), np.abs(uh - uo).max())
    assert (st == so).mean() >= 0.99
    s = dict(zip(["steps", "walks", "capped", "nonfinite", "outside", "inner"], stats.cpu().tolist()))
    assert s["walks"] == pts.shape[1] * wpp and s["steps"] == int(st.sum())


def _gpu_solve(ctx, prob, pts, walks, eps, sb, seed, precision="fp32"):
    acc, stats = ctx.solve(prob, dev(pts), walks, eps, sb, seed=seed, precision=precision)
    m, v, se = (t.cpu().numpy() for t in ctx.finalize(acc))
    return m, se, [int(x) for x in stats.cpu().tolist()], acc


@pytest.mark.parametrize("same_seed", [True, False])
def test_fp32_parity_square2d_full(orc, ctx, same_seed):
    desc = W.square2d_problem()
    pts = W.cell_centres(2, 32)
    sb = orc.sigma_bar(desc)[0]
    prob = ctx.problem(desc)
    m, se, st, _ = _gpu_solve(ctx, prob, pts, 256, 1e-3, sb, seed=0)
    oacc, ost = orc.solve(desc, pts, 256, seed=0 if same_seed else 1, eps=1e-3, sigma_bar=sb)
    om, ov, ose = orc.finalize(oacc)
    ok, nout, mz = four_se_rule(combined_z(m, se, om, ose))
    assert ok, (nout, mz)
    assert st[2] == 0 and st[3] == 0 and st[1] == 1024 * 256
    # steps per walk agree in distribution
    assert abs(st[0] / st[1] - ost["steps"] / ost["walks"]) < 0.05 * ost["steps"] / ost["walks"]


def test_fp32_parity_cube3d_subset(orc, ctx):
    desc = W.cube3d_problem()
    pts = W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 256, 9)]
    sb = orc.sigma_bar(desc, 64)[0]
    prob = ctx.problem(desc)
    m, se, st, _ = _gpu_solve(ctx, prob, pts, 1024, 1e-4, sb, seed=2)
    oacc, _ = orc.solve(desc, pts, 1024, seed=3, eps=1e-4, sigma_bar=sb)
    om, ov, ose = orc.finalize(oacc)
    ok, nout, mz = four_se_rule(combined_z(m, se, om, ose))
    assert ok, (nout, mz)


@pytest.mark.parametrize("name", ["noise_annulus", "noise_cube", "rounded_box", "mesh"])
def test_fp32_parity_other_domains_and_grids(orc, ctx, name):
    mk, ptsf, eps = REPLAY_CASES[name]
    desc = mk()
    pts = ptsf()
    sb = orc.sigma_bar(desc, 64 if desc["dim"] == 3 else 128)[0]
    prob = ctx.problem(desc)
    m, se, st, _ = _gpu_solve(ctx, prob, pts, 2048, eps, sb, seed=4)
    oacc, _ = orc.solve(desc, pts, 2048, seed=5, eps=eps, sigma_bar=sb)
    om, ov, ose = orc.finalize(oacc)
    ok, nout, mz = four_se_rule(combined_z(m, se, om, ose))
    assert ok, (name, nout, mz)


def test_rms_square2d_at_2e16_walks(orc, ctx):
    desc = W.square2d_problem()
    pts = W.cell_centres(2, 32)
    sb = orc.sigma_bar(desc)[0]
    m, se, st, _ = _gpu_solve(ctx, ctx.problem(desc), pts, 1 << 16, 1e-3, sb, seed=11)
    exact = W.square2d_exact(*pts.astype(np.float64))
    assert normalised_rms(m, exact) <= 1e-2
    assert st[2] == 0 and st[3] == 0


def test_rms_cube3d_at_2e16_walks(orc, ctx):
    desc = W.cube3d_problem()
    pts = W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 4096, 12)]
    sb = orc.sigma_bar(desc, 64)[0]
    m, se, st, _ = _gpu_solve(ctx, ctx.problem(desc), pts, 1 << 16, 1e-4, sb, seed=12)
    exact = W.cube3d_exact(*pts.astype(np.float64))
    assert normalised_rms(m, exact) <= 1e-2
    assert st[2] == 0 and st[3] == 0


def test_full_size_cube3d_sampled_points(orc, ctx):
    """The benchmark's workload and launch: 64^3 points x 1024 walks, seed 0."""
    desc = W.cube3d_problem()
    pts = W.cell_centres(3, 64)
    sb = orc.sigma_bar(desc, 64)[0]
    m, se, st, _ = _gpu_solve(ctx, ctx.problem(desc), pts, 1024, 1e-4, sb, seed=0)
    assert st[1] == 64 ** 3 * 1024 and st[2] == 0 and st[3] == 0 and st[4] == 0
    idx = W.seeded_subset(64 ** 3, 24, 13)
    oacc, _ = orc.solve(desc, pts[:, idx], 1024, seed=1, eps=1e-4, sigma_bar=sb)
    om, ov, ose = orc.finalize(oacc)
    ok, nout, mz = four_se_rule(combined_z(m[idx], se[idx], om, ose))
    assert ok, (nout, mz)
    # every point: estimate within 5 standard errors of the exact solution, bar a few
    exact = W.cube3d_exact(*pts.astype(np.float64))
    z = (m - exact) / se
    assert np.mean(np.abs(z) > 5) < 5e-4
    assert abs(np.mean(z)) < 0.05


def test_sigma_bar_matches_oracle(orc, ctx):
    for desc, m in ((W.square2d_problem(), 256), (W.cube3d_problem(), 64), (W.noise_annulus_problem(), 128)):
        got = ctx.sigma_bar(ctx.problem(desc), m)
        want = orc.sigma_bar(desc, m)
        assert np.allclose(got, want, rtol=1e-9, atol=1e-9)


def test_edge_cases(wos, orc, ctx):
    desc = W.square2d_problem()
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc)[0]
    # empty input and zero walks are no-ops
    acc = ctx.new_accum(4)
    ctx.solve(prob, torch.zeros((2, 0), dtype=torch.float32, device="cuda"), 16, 1e-3, sb)
    ctx.solve(prob, dev(W.cell_centres(2, 2)), 0, 1e-3, sb, accum=acc)
    assert int(acc[2].sum()) == 0
    # ragged: 1000 points x 37 walks (not multiples of the warp or the claim chunk)
    pts = W.uniform_in_box(2, 1000, 0.01, 0.99, 14)
    acc, st = ctx.solve(prob, dev(pts), 37, 1e-3, sb, seed=3)
    assert (acc[2].cpu().numpy() == 37).all() and int(st[1]) == 37000
    # per-point walk counts with zeros
    walks = np.array([0, 5, 1, 0, 300, 7] * 50, dtype=np.int32)
    pts = W.uniform_in_box(2, len(walks), 0.05, 0.95, 15)
    acc, st = ctx.solve(prob, dev(pts), torch.from_numpy(walks).cuda(), 1e-3, sb, seed=4)
    assert np.array_equal(acc[2].cpu().numpy(), walks) and int(st[1]) == walks.sum()
    # walk-id continuation: walks 8..15 of one call are walks 0..7 of a call at offset 8
    pts = W.uniform_in_box(2, 20, 0.05, 0.95, 16)
    a, _, _ = ctx.walk_estimates(prob, dev(pts), 16, 1e-3, sb, seed=5, precision="fp64")
    b, _, _ = ctx.walk_estimates(prob, dev(pts), 8, 1e-3, sb, seed=5, walk_offset=8, precision="fp64")
    assert torch.equal(a[:, 8:], b)
    # accumulating two calls equals counting both
    acc = ctx.new_accum(20)
    ctx.solve(prob, dev(pts), 10, 1e-3, sb, seed=6, accum=acc)
    ctx.solve(prob, dev(pts), 10, 1e-3, sb, seed=6, walk_offset=10, accum=acc)
    assert (acc[2].cpu().numpy() == 20).all()
    # points in the epsilon shell return g at the closest point, zero variance
    pts = np.array([[0.5, 2e-4, 0.3], [0.9995, 0.5, 1 - 1e-4]], dtype=np.float32)
    m, se, st, _ = _gpu_solve(ctx, prob, pts, 9, 1e-3, sb, seed=7)
    want = [W.square2d_exact(*orc.distance(desc, pts[:, i].astype(np.float64))[1]) for i in range(3)]
    # every walk returns the same value: the spread is rounding of the FP64 sums only
    assert np.allclose(m, want, rtol=1e-6) and np.all(se <= 1e-7 * np.abs(m) + 1e-12) and st[0] == 0
    # invalid arguments are rejected with WOS_EINVAL
    for kw in ({"eps": 0.0}, {"eps": -1.0}, {"sigma_bar": 0.0}, {"sigma_bar": float("nan")},
               {"max_steps": 0}):
        args = {"eps": 1e-3, "sigma_bar": sb, "max_steps": 1 << 20}
        args.update(kw)
        with pytest.raises(wos.WosError) as e:
            ctx.solve(prob, dev(pts), 4, args["eps"], args["sigma_bar"], max_steps=args["max_steps"])
        assert e.value.code == wos.WOS_EINVAL
    bad = W.square2d_problem()
    bad["dim"] = 4
    with pytest.raises(wos.WosError):
        ctx.problem(bad)
    bad = W.square2d_problem()
    bad["alpha"] = W.const(-1.0)
    with pytest.raises(wos.WosError):
        ctx.problem(bad)
    bad = W.noise_cube_problem()
    bad["alpha"]["kind"] = "grid_linear"
    with pytest.raises(wos.WosError):
        ctx.problem(bad)
    # step cap: counted, never hidden
    _, st = ctx.solve(prob, dev(W.cell_centres(2, 4)), 50, 1e-3, sb, max_steps=2)
    st = [int(x) for x in st.cpu().tolist()]
    assert st[2] > 0 and st[0] <= 2 * st[1]


def test_solve_host_matches_device(orc, ctx):
    desc = W.cube3d_problem()
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc, 64)[0]
    pts = W.cell_centres(3, 16)
    m_d, se_d, _, _ = _gpu_solve(ctx, prob, pts, 64, 1e-4, sb, seed=9)
    mean, var, se, stats = ctx.solve_host(prob, pts, 64, 1e-4, sb, seed=9)
    assert np.allclose(mean.numpy(), m_d, rtol=1e-12, atol=1e-12)
    assert np.allclose(se.numpy(), se_d, rtol=1e-9, atol=1e-12)
    assert int(stats[1]) == 16 ** 3 * 64


def test_mesh_noise_workload_sampled_points(orc, ctx):
    """Displaced icosphere (327,680 triangles) with 128^3 noise grids: FP32 GPU against the
    oracle on sampled interior points, and the manufactured solution on the same mesh."""
    desc = W.mesh_noise_problem(level=7)
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc, 48)[0]
    assert ctx.sigma_bar(prob, 48) == pytest.approx(orc.sigma_bar(desc, 48), rel=1e-9)
    pts = W.mesh_interior_points(12, seed=8)
    m, se, st, _ = _gpu_solve(ctx, prob, pts, 1024, 1e-4, sb, seed=3)
    oacc, _ = orc.solve(desc, pts, 512, seed=4, eps=1e-4, sigma_bar=sb)
    om, ov, ose = orc.finalize(oacc)
    ok, nout, mz = four_se_rule(combined_z(m, se, om, ose))
    assert ok, (nout, mz)
    assert st[2] == 0 and st[3] == 0
    man = W.mesh_manufactured_problem(level=7)
    mp = ctx.problem(man)
    sbm = orc.sigma_bar(man, 48)[0]
    pts = W.mesh_interior_points(2048, seed=9)
    m, se, st, _ = _gpu_solve(ctx, mp, pts, 1 << 14, 1e-4, sbm, seed=5)
    exact = W.cube3d_exact(*pts.astype(np.float64))
    ok, nout, mz = four_se_rule((m - exact) / se)
    assert ok, (nout, mz)


@pytest.mark.parametrize("name", ["square2d", "cube3d", "hifreq"])
def test_weight_window_fp64_replay_and_fp32_parity(orc, ctx, name):
    if name == "hifreq":
        desc, pts, eps = W.hifreq_alpha_problem(), W.cell_centres(2, 8)[:, ::3], 1e-3
    else:
        mk, ptsf, eps = REPLAY_CASES[name]
        desc, pts = mk(), ptsf()[:, :24]
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc, 64 if desc["dim"] == 3 else 128)[0]
    win = (0.5, 1.5, 8)
    uh, st, _ = ctx.walk_estimates(prob, dev(pts), 8, eps, sb, seed=17, precision="fp64", window=win)
    uh = uh.cpu().numpy()
    st = st.cpu().numpy()
    pk = orc.pack(desc)
    ok, steps_ok, n = 0, 0, 0
    for i in range(pts.shape[1]):
        for j in range(8):
            u, k, _ = orc.walk_ww(desc, pts[:, i].astype(np.float64), i, j, 17, eps, sb, 0.5, 1.5, 8, packed=pk)
            ok += abs(uh[i, j] - u) <= 1e-9 * max(1.0, abs(u))
            steps_ok += st[i, j] == k
            n += 1
    assert ok >= 0.99 * n and steps_ok >= 0.99 * n, (ok, steps_ok, n)
    m, se, s, _ = (lambda a: (ctx.finalize(a[0])[0].cpu().numpy(), ctx.finalize(a[0])[2].cpu().numpy(),
                              [int(v) for v in a[1].cpu().tolist()], a[0]))(
        ctx.solve(prob, dev(pts), 2048, eps, sb, seed=18, window=win))
    oacc, _ = orc.solve_ww(desc, pts, 2048, seed=19, eps=eps, sigma_bar=sb, ww_lo=0.5, ww_hi=1.5)
    om, ov, ose = orc.finalize(oacc)
    good, nout, mz = four_se_rule(combined_z(m, se, om, ose))
    assert good, (nout, mz)


def test_fp32_matches_finite_difference_solve(ctx, orc):
    """No closed-form solution: FP32 walks at 2^16 per point against a second-order
    finite-difference solve of eq. 1 (N = 256) on 15^2 grid nodes."""
    from tests.fd_reference import fd_reference_at
    desc = W.fd_square_problem()
    g = np.arange(1, 16) / 16.0
    pts = np.array(np.meshgrid(g, g, indexing="ij")).reshape(2, -1)
    want = fd_reference_at(W.fd_square_coefficients(), pts, n=256)
    sb = orc.sigma_bar(desc)[0]
    prob = ctx.problem(desc)
    m, se, st, _ = _gpu_solve(ctx, prob, pts, 1 << 16, 1e-4, sb, seed=3)
    ok, nout, mz = four_se_rule((m - want) / se)
    assert ok, (nout, mz)
    assert normalised_rms(m, want) <= 1e-2


def _csg_inside(orc, prob, n, seed, margin=0.02):
    dim = prob["dim"]
    lo = np.array(prob["domain"]["p"][:dim])
    hi = np.array(prob["domain"]["p"][3:3 + dim])
    X = lo + (hi - lo) * np.random.default_rng(seed).uniform(size=(8 * n + 4000, dim))
    d = np.array([orc.distance(prob, x)[0] for x in X])
    return np.ascontiguousarray(X[d > margin][:n].T.astype(np.float32))


@pytest.mark.parametrize("name", ["csg2d", "csg3d", "csg_variable"])
def test_csg_fp64_replay_and_fp32_parity(orc, ctx, name):
    """Signed-distance CSG domains (Sec. 7.2): FP64 walks replay the oracle's per walk; FP32
    estimates agree with the exact solution within 4 standard errors."""
    desc = {"csg2d": lambda: W.csg_laplace_problem(2), "csg3d": lambda: W.csg_laplace_problem(3),
            "csg_variable": W.csg_variable_problem}[name]()
    pts = _csg_inside(orc, desc, 48, seed=11)
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc)[0]
    uh, st, _ = ctx.walk_estimates(prob, dev(pts), 16, 1e-4, sb, seed=3, precision="fp64")
    uo, so = orc.walks(desc, pts, 16, seed=3, eps=1e-4, sigma_bar=sb)
    ok = np.abs(uh.cpu().numpy() - uo) <= 1e-9 * np.maximum(1.0, np.abs(uo))
    assert ok.mean() >= 0.99 and (st.cpu().numpy() == so).mean() >= 0.99
    m, se, s, _ = _gpu_solve(ctx, prob, pts, 8192, 1e-4, sb, seed=4)
    p64 = pts.astype(np.float64)
    exact = W.cube3d_exact(*p64) if name == "csg_variable" else W.csg_laplace_exact(desc["dim"], p64)
    ok, nout, mz = four_se_rule((m - exact) / se)
    assert ok, (nout, mz)
    assert s[2] == 0 and s[4] == 0


def test_mesh_distance_grid_fp32_exact_solution(orc, ctx):
    """Mesh walks with the distance grid (radius: the grid's Lipschitz lower bound away from
    the boundary), alone and with certified radii near the boundary, against the manufactured
    solution, and their step count against exact radii."""
    pts = W.mesh_interior_points(128, 13)
    exact = W.cube3d_exact(*pts.astype(np.float64))
    res = {}
    for grid, tol in ((0, 0.0), (64, 0.0), (64, 0.1)):
        desc = W.mesh_manufactured_problem(level=6, dist_grid=grid, tol=tol)
        prob = ctx.problem(desc)
        sb = orc.sigma_bar(desc, 48)[0]
        m, se, st, _ = _gpu_solve(ctx, prob, pts, 4096, 1e-4, sb, seed=8)
        ok, nout, mz = four_se_rule((m - exact) / se)
        assert ok, (grid, tol, nout, mz)
        res[(grid, tol)] = st[0] / st[1]
    assert res[(64, 0.0)] < 1.2 * res[(0, 0.0)]
    # the grid with certified radii near the boundary (both lower bounds of the distance)
    assert res[(64, 0.1)] < 1.4 * res[(0, 0.0)]


@pytest.mark.parametrize("tol", [0.1, 0.25])
def test_mesh_tolerance_walk_matches_the_exact_walk(orc, ctx, tol):
    """Distance queries that stop at a certified radius (1 - tol) d <= r <= d: FP32 GPU walks on
    the 327,680-triangle noise workload against the oracle's exact-radius walks (4 combined
    standard errors; any ball inside the domain keeps the estimator unbiased), and against
    the manufactured solution on the same mesh; the query counters are reported and no
    search is exhausted."""
    desc = W.mesh_noise_problem(level=7, tol=tol)
    prob = ctx.problem(desc)
    exact_desc = W.mesh_noise_problem(level=7)
    sb = orc.sigma_bar(exact_desc, 48)[0]
    pts = W.mesh_interior_points(12, seed=18)
    m, se, st, _ = _gpu_solve(ctx, prob, pts, 1024, 1e-4, sb, seed=13)
    oacc, _ = orc.solve(exact_desc, pts, 512, seed=14, eps=1e-4, sigma_bar=sb)
    om, ov, ose = orc.finalize(oacc)
    ok, nout, mz = four_se_rule(combined_z(m, se, om, ose))
    assert ok, (nout, mz)
    assert st[2] == 0 and st[3] == 0 and st[8] == 0
    assert st[6] > 0 and st[7] > 0  # nodes and triangles of the queries
    man = W.mesh_manufactured_problem(level=7, tol=tol)
    mp = ctx.problem(man)
    sbm = orc.sigma_bar(W.mesh_manufactured_problem(level=7), 48)[0]
    pts = W.mesh_interior_points(2048, seed=19)
    m, se, st, _ = _gpu_solve(ctx, mp, pts, 1 << 14, 1e-4, sbm, seed=15)
    exact = W.cube3d_exact(*pts.astype(np.float64))
    ok, nout, mz = four_se_rule((m - exact) / se)
    assert ok, (nout, mz)
    assert st[8] == 0


def test_mesh_tolerance_cuts_query_work(wos, orc, ctx):
    """The same walks' distance queries open fewer BVH nodes and test far fewer triangles per
    step with tol = 0.1 than with exact radii."""
    pts = dev(W.mesh_interior_points(4096, seed=20))
    per = {}
    for tol in (0.0, 0.1):
        desc = W.mesh_noise_problem(level=7, tol=tol)
        prob = ctx.problem(desc)
        acc, stats = ctx.solve(prob, pts, 16, 1e-4, 787.0, seed=21)
        s = wos.stats_dict(stats)
        per[tol] = (s["mesh_nodes"] / s["steps"], s["mesh_tris"] / s["steps"], s["steps"] / s["walks"])
        assert s["exhausted"] == 0
    assert per[0.1][0] < 0.5 * per[0.0][0] and per[0.1][1] < 0.2 * per[0.0][1], per
    assert per[0.1][2] < 1.5 * per[0.0][2], per  # balls at least 0.9 d: a few more steps per walk
