"""GPU parity of the problem-specialised walk kernels (runtime compilation) with the oracle.

A specialised kernel is the walk kernel compiled for one problem, with the problem's
fields written out as code; every solve on a specialised problem launches it.

* FP64 replay: per walk, equal to the oracle's walk on the same Philox streams
  (>= 99% of walks to 1e-9 of max(1, |u|), equal step counts), for analytic, grid,
  mesh, CSG and extra-drift problems, and for the gradient and weight-window variants.
* FP32: per walk against the generic FP32 kernel on the same streams (the two
  differ only in the rounding of the field arithmetic), and the full-size 3D
  workload in the benchmark's launch against the exact solution.
* The API: which kernels are loaded, unknown flags, variants a problem cannot run.
"""
import numpy as np
import pytest

import workloads as W
from tests.stats_util import four_se_rule
from tests.test_jit import GRID_DESC, all_atoms_problem

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


def _csg_points(orc, desc, n=32, seed=11, margin=0.02):
    dim = desc["dim"]
    lo = np.array(desc["domain"]["p"][:dim])
    hi = np.array(desc["domain"]["p"][3:3 + dim])
    X = lo + (hi - lo) * np.random.default_rng(seed).uniform(size=(8 * n + 4000, dim))
    d = np.array([orc.distance(desc, x)[0] for x in X])
    return np.ascontiguousarray(X[d > margin][:n].T.astype(np.float32))


# name: (problem, points(orc, desc), eps)
CASES = {
    "cube3d": (W.cube3d_problem, lambda o, d: W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 48, 2)], 1e-4),
    "square2d": (W.square2d_problem, lambda o, d: W.cell_centres(2, 32)[:, W.seeded_subset(1024, 48, 1)], 1e-3),
    "hifreq": (W.hifreq_alpha_problem, lambda o, d: W.cell_centres(2, 16)[:, W.seeded_subset(256, 32, 8)], 1e-3),
    "all_atoms": (all_atoms_problem, lambda o, d: W.uniform_in_box(3, 32, 0.05, 0.95, 3), 1e-4),
    "grids": (GRID_DESC, lambda o, d: W.uniform_in_box(3, 32, 0.05, 0.95, 9), 1e-4),
    "mesh": (lambda: W.mesh_manufactured_problem(level=5), lambda o, d: W.mesh_interior_points(32, 7), 1e-4),
    "csg": (W.csg_variable_problem, _csg_points, 1e-4),
    "drift": (W.cube3d_literal_problem, lambda o, d: W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 32, 5)],
              1e-4),
}


def _sb(orc, desc):
    return orc.sigma_bar(desc, 64 if desc["dim"] == 3 else 128)[0]


@pytest.mark.parametrize("name", list(CASES))
def test_specialised_fp64_replay_per_walk(orc, ctx, wos, name):
    mk, ptsf, eps = CASES[name]
    desc = mk()
    pts = ptsf(orc, desc)
    prob = ctx.problem(desc, specialize=(("fp64",), ("plain",)))
    assert prob.specialized() == wos.WOS_SPEC_FP64 | wos.WOS_SPEC_PLAIN
    sb = _sb(orc, desc)
    uh, st, stats = ctx.walk_estimates(prob, dev(pts), 16, eps, sb, seed=7, precision="fp64")
    uo, so = orc.walks(desc, pts, 16, seed=7, eps=eps, sigma_bar=sb)
    uh, st = uh.cpu().numpy(), st.cpu().numpy()
    ok = np.abs(uh - uo) <= 1e-9 * np.maximum(1.0, np.abs(uo))
    assert ok.mean() >= 0.99, (name, ok.mean(), np.nanmax(np.abs(uh - uo)))
    assert (st == so).mean() >= 0.99
    s = wos.stats_dict(stats)
    assert s["walks"] == pts.shape[1] * 16 and s["steps"] == int(st.sum())


@pytest.mark.parametrize("name", ["cube3d", "square2d", "all_atoms", "grids", "mesh", "drift"])
def test_specialised_fp32_equals_generic_fp32_per_walk(orc, ctx, name):
    mk, ptsf, eps = CASES[name]
    desc = mk()
    pts = ptsf(orc, desc)
    sb = _sb(orc, desc)
    gen = ctx.problem(desc)
    spec = ctx.problem(desc, specialize=(("fp32",), ("plain",)))
    ug, sg, _ = ctx.walk_estimates(gen, dev(pts), 32, eps, sb, seed=3)
    us, ss, _ = ctx.walk_estimates(spec, dev(pts), 32, eps, sb, seed=3)
    ug, us = ug.cpu().numpy(), us.cpu().numpy()
    ok = np.abs(us - ug) <= 1e-3 * np.maximum(1.0, np.abs(ug))
    assert ok.mean() >= 0.97, (name, ok.mean())
    assert (ss.cpu().numpy() == sg.cpu().numpy()).mean() >= 0.97


@pytest.mark.parametrize("name", ["cube3d", "square2d", "grids"])
def test_specialised_gradient_fp64_replay(orc, ctx, wos, name):
    mk, ptsf, eps = CASES[name]
    desc = mk()
    pts = ptsf(orc, desc)[:, :24]
    prob = ctx.problem(desc, specialize=(("fp64",), ("grad",)))
    sb = _sb(orc, desc)
    uh, gh, st, _ = ctx.walk_grad_estimates(prob, dev(pts), 16, eps, sb, seed=5, precision="fp64")
    uo, go, so = orc.walks_grad(desc, pts, 16, seed=5, eps=eps, sigma_bar=sb)
    uh, gh = uh.cpu().numpy(), gh.cpu().numpy()
    ok_u = np.abs(uh - uo) <= 1e-9 * np.maximum(1.0, np.abs(uo))
    scale = np.maximum(1.0, np.sqrt(np.sum(go ** 2, axis=0)))
    ok_g = np.all(np.abs(gh - go) <= 1e-8 * scale[None], axis=0)
    assert (ok_u & ok_g).mean() >= 0.99, (name, ok_u.mean(), ok_g.mean())


@pytest.mark.parametrize("name", ["cube3d", "square2d"])
def test_specialised_weight_window_fp64_replay(orc, ctx, name):
    mk, ptsf, eps = CASES[name]
    desc = mk()
    pts = ptsf(orc, desc)[:, :16]
    prob = ctx.problem(desc, specialize=(("fp64",), ("window",)))
    sb = _sb(orc, desc)
    uh, st, _ = ctx.walk_estimates(prob, dev(pts), 8, eps, sb, seed=17, precision="fp64", window=(0.5, 1.5, 8))
    uh, st = uh.cpu().numpy(), st.cpu().numpy()
    pk = orc.pack(desc)
    ok, n = 0, 0
    for i in range(pts.shape[1]):
        for j in range(8):
            u, k, _ = orc.walk_ww(desc, pts[:, i].astype(np.float64), i, j, 17, eps, sb, 0.5, 1.5, 8, packed=pk)
            ok += abs(uh[i, j] - u) <= 1e-9 * max(1.0, abs(u)) and st[i, j] == k
            n += 1
    assert ok >= 0.99 * n, (ok, n)


def test_specialised_full_size_cube3d(orc, ctx):
    """The benchmark's workload and launch (64^3 points x 1024 walks, seed 0) through the
    specialised kernel: every point within 5 standard errors of the exact solution bar a few."""
    desc = W.cube3d_problem()
    pts = W.cell_centres(3, 64)
    sb = orc.sigma_bar(desc, 64)[0]
    prob = ctx.problem(desc, specialize=(("fp32",), ("plain",)))
    acc, stats = ctx.solve(prob, dev(pts), 1024, 1e-4, sb, seed=0)
    m, v, se = (t.cpu().numpy() for t in ctx.finalize(acc))
    s = [int(x) for x in stats.cpu().tolist()]
    assert s[1] == 64 ** 3 * 1024 and s[2] == 0 and s[3] == 0 and s[4] == 0
    z = (m - W.cube3d_exact(*pts.astype(np.float64))) / se
    assert np.mean(np.abs(z) > 5) < 5e-4 and abs(np.mean(z)) < 0.05
    idx = W.seeded_subset(64 ** 3, 4096, 3)
    ok, nout, mz = four_se_rule(z[idx])
    assert ok, (nout, mz)


def test_specialisation_api(orc, ctx, wos):
    desc = W.cube3d_problem()
    prob = ctx.problem(desc)
    assert prob.specialized() == 0
    prob.specialize(("fp32",), ("plain", "grad"))
    assert prob.specialized() == wos.WOS_SPEC_FP32 | wos.WOS_SPEC_PLAIN | wos.WOS_SPEC_GRAD
    prob.specialize(("fp32",), ("plain",))  # already loaded: no recompilation
    assert prob.specialized() == wos.WOS_SPEC_FP32 | wos.WOS_SPEC_PLAIN | wos.WOS_SPEC_GRAD
    rc = ctx.lib.wos_problem_specialize(ctx.handle, prob.handle, 0x1000)
    assert rc == wos.WOS_EINVAL
    drift = ctx.problem(W.cube3d_literal_problem())
    with pytest.raises(wos.WosError) as e:
        drift.specialize(("fp32",), ("window",))
    assert e.value.code == wos.WOS_EUNSUPPORTED
    # the other entry points of a specialised problem keep working (generic kernels)
    sb = orc.sigma_bar(desc, 64)[0]
    pts = dev(W.cell_centres(3, 8))
    acc, st = ctx.solve_nf(prob, pts, 4, 1e-4, sb)
    assert wos.stats_dict(st)["walks"] == 8 ** 3 * 4
    prob.close()
    drift.close()
