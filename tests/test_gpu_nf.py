"""GPU parity of the next-flight walks (Sec. 5.2, Supplemental Algorithm 2) with the oracle.

* FP64 replay: per walk, the kernel's estimate and ball count equal the oracle's
  on the same Philox streams (>= 99% of walks, 1e-9 relative to max(1, |u|)).
* FP32: per walk against the FP64 kernel on the same streams (the roulette and
  shell decisions agree except for rare rounding flips), and against the exact
  solution where the next-flight estimate is exact (sigma_bar = sigma').
* Counters: balls (distance queries) and inner iterations.
* The series kernels (series_terms > 0): the same FP64 per-walk replay against the
  oracle's series walk, and the FP32 estimate against the exact solution where sigma'
  varies (the printed approximations are biased there).
"""
import numpy as np
import pytest

import workloads as W
from tests.stats_util import four_se_rule

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


CASES = {
    "square2d": (W.square2d_problem, lambda: W.cell_centres(2, 32)[:, W.seeded_subset(1024, 48, 1)], 1e-3, None),
    "cube3d": (W.cube3d_problem, lambda: W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 48, 2)], 1e-4, None),
    "hifreq": (W.hifreq_alpha_problem, lambda: W.cell_centres(2, 16)[:, W.seeded_subset(256, 32, 8)], 1e-3, None),
    "screened_ball": (W.screened_ball_problem, lambda: W.uniform_in_ball(3, 48, [0, 0, 0], 1.0, 4, 0.02), 1e-4,
                      9.0),
    "laplace_disk": (W.laplace_disk_problem, lambda: W.uniform_in_ball(2, 48, [0, 0], 1.0, 3, 0.02), 1e-4, None),
    "mesh": (lambda: W.mesh_manufactured_problem(level=5), lambda: W.mesh_interior_points(32, 7), 1e-4, None),
}


def _sb(orc, desc, sb):
    return sb if sb is not None else orc.sigma_bar(desc, 64 if desc["dim"] == 3 else 128)[0]


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_replay_next_flight_per_walk(orc, ctx, wos, name):
    mk, ptsf, eps, sb = CASES[name]
    desc = mk()
    pts = ptsf()
    prob = ctx.problem(desc)
    sb = _sb(orc, desc, sb)
    wpp = 16
    uh, st, stats = ctx.walk_estimates_nf(prob, dev(pts), wpp, eps, sb, seed=9, precision="fp64", series_terms=0)
    uo, so, io = orc.walks_nf(desc, pts, wpp, seed=9, eps=eps, sigma_bar=sb)
    uh, st = uh.cpu().numpy(), st.cpu().numpy()
    ok = np.abs(uh - uo) <= 1e-9 * np.maximum(1.0, np.abs(uo))
    assert ok.mean() >= 0.99, (name, ok.mean())
    assert (st == so).mean() >= 0.99
    s = wos.stats_dict(stats)
    assert s["walks"] == pts.shape[1] * wpp and s["steps"] == int(st.sum())
    # inner iterations: equal to the oracle's when every walk replays
    if ok.all() and (st == so).all():
        assert s["inner"] == int(io.sum())


@pytest.mark.parametrize("nser", [0, 8])
@pytest.mark.parametrize("name", ["square2d", "cube3d", "screened_ball", "mesh"])
def test_fp32_next_flight_matches_fp64_per_walk(orc, ctx, name, nser):
    mk, ptsf, eps, sb = CASES[name]
    desc = mk()
    pts = ptsf()
    prob = ctx.problem(desc)
    sb = _sb(orc, desc, sb)
    u64, s64, _ = ctx.walk_estimates_nf(prob, dev(pts), 32, eps, sb, seed=2, precision="fp64", series_terms=nser)
    u32, s32, _ = ctx.walk_estimates_nf(prob, dev(pts), 32, eps, sb, seed=2, precision="fp32", series_terms=nser)
    u64, u32 = u64.cpu().numpy(), u32.cpu().numpy()
    ok = np.abs(u32 - u64) <= 1e-3 * np.maximum(1.0, np.abs(u64))
    assert ok.mean() >= 0.95, (name, ok.mean())


@pytest.mark.parametrize("name,sb", [("screened_ball", 9.0), ("screened_square", 4.0)])
def test_fp32_next_flight_exact_when_sigma_bar_is_sigma(ctx, name, sb):
    if name == "screened_ball":
        desc = W.screened_ball_problem()
        pts = W.uniform_in_ball(3, 256, [0, 0, 0], 1.0, 6, 0.02)
        exact = W.screened_ball_exact(9.0, *pts.astype(np.float64))
    else:
        desc = W.screened_square_problem()
        pts = W.uniform_in_box(2, 256, 0.02, 0.98, 7)
        exact = W.screened_square_exact(*pts.astype(np.float64))
    prob = ctx.problem(desc)
    for nser in (0, 8):
        acc, stats = ctx.solve_nf(prob, dev(pts), 4096, 1e-4, sb, seed=1, series_terms=nser)
        m, v, se = (t.cpu().numpy() for t in ctx.finalize(acc))
        ok, nout, mz = four_se_rule((m - exact) / se)
        assert ok, (nser, nout, mz)


@pytest.mark.parametrize("name", ["square2d", "cube3d", "hifreq", "screened_ball", "mesh"])
def test_fp64_replay_next_flight_series_per_walk(orc, ctx, wos, name):
    mk, ptsf, eps, sb = CASES[name]
    desc = mk()
    pts = ptsf()
    prob = ctx.problem(desc)
    sb = _sb(orc, desc, sb)
    wpp, nser = 8, 12
    uh, st, stats = ctx.walk_estimates_nf(prob, dev(pts), wpp, eps, sb, seed=5, precision="fp64", series_terms=nser)
    uo, so, io = orc.walks_nf(desc, pts, wpp, seed=5, eps=eps, sigma_bar=sb, series_terms=nser)
    uh, st = uh.cpu().numpy(), st.cpu().numpy()
    ok = np.abs(uh - uo) <= 1e-9 * np.maximum(1.0, np.abs(uo))
    assert ok.mean() >= 0.99, (name, ok.mean())
    assert (st == so).mean() >= 0.99


@pytest.mark.parametrize("name", ["cube3d", "square2d"])
def test_fp32_next_flight_series_is_unbiased_where_sigma_varies(orc, ctx, wos, name):
    if name == "cube3d":
        desc, exact = W.cube3d_problem(), W.cube3d_exact
        pts = W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 256, 3)]
        sb = orc.sigma_bar(desc, 64)[0]
    else:
        desc, exact = W.square2d_problem(), W.square2d_exact
        pts = W.cell_centres(2, 32)[:, W.seeded_subset(1024, 256, 4)]
        sb = orc.sigma_bar(desc)[0]
    prob = ctx.problem(desc)
    acc, stats = ctx.solve_nf(prob, dev(pts), 16384, 1e-4, sb, seed=3, series_terms=8)
    m, v, se = (t.cpu().numpy() for t in ctx.finalize(acc))
    ex = np.array([exact(*pts[:, i].astype(np.float64)) for i in range(pts.shape[1])])
    ok, nout, mz = four_se_rule((m - ex) / se)
    assert ok, (name, nout, mz)
    assert wos.stats_dict(stats)["nonfinite"] == 0


def test_next_flight_arguments(ctx, orc, wos):
    desc = W.square2d_problem()
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc)[0]
    pts = dev(W.cell_centres(2, 4))
    with pytest.raises(wos.WosError):
        ctx.solve_nf(prob, pts, 8, 1e-3, sb, max_inner=0)
    for bad in (-1, 65):
        with pytest.raises(wos.WosError):
            ctx.solve_nf(prob, pts, 8, 1e-3, sb, series_terms=bad)
    acc, st = ctx.solve_nf(prob, pts, 8, 1e-3, sb, max_inner=1)  # every ball cut after one iteration
    s = wos.stats_dict(st)
    assert s["walks"] == 16 * 8 and s["inner"] <= s["steps"]
