"""The problem-statement calls (domain and field handles, wos_problem_assemble,
wos_problem_sigma_bar, wos_solve_mean, wos_solve_batched, wos_adjoint) against the
descriptor entry points they are layered on:

* a problem assembled from handles runs the same walks as the one built from a
  description: FP64 sums agree to summation-order rounding, counts exactly (analytic
  fields with a manufactured source, noise grids, and a mesh given as device arrays);
* the default sigma_bar is wos_sigma_bar on the stated lattice;
* wos_solve_mean equals wos_solve + wos_finalize, and two calls with consecutive walk
  ids merge (Chan et al.) into the estimate of one call with all the walks;
* wos_solve_batched equals a batch created and solved by hand;
* wos_adjoint equals wos_adjoint_sigma and wos_adjoint_alpha rounded to float32;
* an open mesh is rejected.
"""
import numpy as np
import pytest

import workloads as W

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


def domain_handle(ctx, desc):
    dom = desc["domain"]
    dim = desc["dim"]
    if dom["kind"] == "box":
        return ctx.domain_box(dim, dom["p"][:dim], dom["p"][3:3 + dim])
    if dom["kind"] == "mesh":
        v = torch.from_numpy(np.ascontiguousarray(dom["verts"], dtype=np.float32)).cuda()
        t = torch.from_numpy(np.ascontiguousarray(dom["tris"], dtype=np.int32)).cuda()
        return ctx.domain_mesh(v, t)
    n = {"ball": 4, "annulus": 5, "rounded_box": 7}[dom["kind"]]
    return ctx.domain_sdf(dim, dom["kind"], dom["p"][:n])


def assemble(wos, ctx, desc):
    """The same problem built from handles (a manufactured source carries u_m's terms)."""
    dim = desc["dim"]
    f = (ctx.field_analytic("manufactured", wos.pack_terms(desc["um"]["terms"]))
         if desc["f"]["kind"] == "manufactured" else ctx.field(desc["f"], dim))
    phi = None if desc["phi"]["kind"] == "zero" else ctx.field(desc["phi"], dim)
    return ctx.problem_assemble(domain_handle(ctx, desc), ctx.field(desc["alpha"], dim),
                                ctx.field(desc["sigma"], dim), phi, f, ctx.field(desc["g"], dim))


CASES = {
    "cube3d": (W.cube3d_problem, lambda: W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 300, 5)], 1e-4),
    "noise_annulus": (W.noise_annulus_problem,
                      lambda: np.array([[0.5, -0.6, 0.0, 0.7], [0.2, 0.3, -0.8, -0.5]], dtype=np.float32), 1e-3),
    "rounded_box": (W.rounded_box_problem, lambda: W.uniform_in_box(2, 200, -0.3, 0.3, 6), 1e-3),
    "mesh": (lambda: W.mesh_manufactured_problem(level=3), lambda: W.mesh_interior_points(200, 8), 1e-4),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_assembled_problem_runs_the_same_walks(wos, orc, ctx, name):
    make, pts_fn, eps = CASES[name]
    desc = make()
    pts = torch.from_numpy(np.ascontiguousarray(pts_fn(), dtype=np.float32)).cuda()
    ref_prob = ctx.problem(desc)
    got_prob = assemble(wos, ctx, desc)
    sb = ctx.sigma_bar(ref_prob)[0]
    assert ctx.sigma_bar(got_prob)[0] == sb
    ref, _ = ctx.solve(ref_prob, pts, 32, eps, sb, seed=3, precision="fp64")
    got, _ = ctx.solve(got_prob, pts, 32, eps, sb, seed=3, precision="fp64")
    assert torch.equal(ref[2], got[2])
    assert torch.allclose(ref[0], got[0], rtol=1e-11, atol=1e-12)
    assert torch.allclose(ref[1], got[1], rtol=1e-11, atol=1e-12)


def test_default_sigma_bar_is_the_stated_lattice(wos, ctx):
    for desc, m in ((W.cube3d_problem(), 128), (W.square2d_problem(), 256)):
        p = ctx.problem(desc)
        assert ctx.problem_sigma_bar(p) == ctx.sigma_bar(p, m)


def test_solve_mean_equals_finalize_and_merges_calls(wos, ctx):
    desc = W.square2d_problem()
    prob = ctx.problem(desc)
    sb = ctx.sigma_bar(prob)[0]
    pts = torch.from_numpy(W.cell_centres(2, 16)).cuda()
    acc, _ = ctx.solve(prob, pts, 96, 1e-3, sb, seed=9, precision="fp64")
    mean, var, _ = ctx.finalize(acc)
    one, _ = ctx.solve_mean(prob, pts, 96, 1e-3, sb, seed=9, precision="fp64")
    assert torch.equal(one[2], acc[2])
    assert torch.allclose(one[0], mean, rtol=1e-11, atol=1e-12)
    assert torch.allclose(one[1], var, rtol=1e-9, atol=1e-12)
    # 40 + 56 walks with consecutive walk ids, merged, equal the 96 walks of one call
    two, _ = ctx.solve_mean(prob, pts, 40, 1e-3, sb, seed=9, precision="fp64")
    two, _ = ctx.solve_mean(prob, pts, 56, 1e-3, sb, seed=9, walk_offset=40, precision="fp64", moments=two)
    assert torch.equal(two[2], acc[2])
    assert torch.allclose(two[0], mean, rtol=1e-10, atol=1e-12)
    assert torch.allclose(two[1], var, rtol=1e-8, atol=1e-12)
    # per-point walk counts, some zero: those points keep their entry values
    w = torch.from_numpy(np.random.default_rng(2).integers(0, 4, size=pts.shape[1]).astype(np.int32)).cuda()
    mom = ctx.new_moments(pts.shape[1])
    mom[0].fill_(7.0)
    ctx.solve_mean(prob, pts, w, 1e-3, sb, seed=9, precision="fp64", moments=mom)
    zero = (w == 0)
    assert torch.equal(mom[2], w.to(torch.int64))
    assert bool((mom[0][zero] == 7.0).all())


def test_solve_batched_equals_a_batch(wos, orc, ctx):
    probs, pts, offs, walks = W.batch_problems(12, seed=5, max_points=40, min_points=4, min_walks=8, max_walks=32)
    sbs = np.array([orc.sigma_bar(p, 96)[0] for p in probs])
    hp = [ctx.problem(p) for p in probs]
    p = torch.from_numpy(pts).cuda()
    w = torch.from_numpy(walks).cuda()
    batch = ctx.batch(hp, offs, sbs)
    acc, _ = ctx.solve_batch(batch, p, w, 1e-3, seed=17, precision="fp64")
    mean, var, _ = ctx.finalize(acc)
    got, _ = ctx.solve_batched(hp, offs, sbs, p, w, 1e-3, seed=17, precision="fp64")
    assert torch.equal(got[2], acc[2])
    assert torch.allclose(got[0], mean, rtol=1e-11, atol=1e-12)
    assert torch.allclose(got[1], var, rtol=1e-9, atol=1e-12)
    # sigma_bars NULL: each problem's default bound
    own = np.array([ctx.problem_sigma_bar(q)[0] for q in hp])
    acc2, _ = ctx.solve_batch(ctx.batch(hp, offs, own), p, 8, 1e-3, seed=18, precision="fp64")
    m2, _, _ = ctx.finalize(acc2)
    got2, _ = ctx.solve_batched(hp, offs, None, p, 8, 1e-3, seed=18, precision="fp64")
    assert torch.allclose(got2[0], m2, rtol=1e-11, atol=1e-12)


def test_combined_adjoint_equals_the_two_replays(wos, orc, ctx):
    sg = W.inverse_sigma_grid()
    desc = W.inverse_problem(sg)
    prob = ctx.problem(desc)
    sb = ctx.sigma_bar(prob)[0]
    pts = torch.from_numpy(W.inverse_sensors(256, 4)).cuda()
    gu = torch.from_numpy(np.random.default_rng(3).normal(size=256)).cuda()
    ns, na = sg.size, W.inverse_alpha_grid().size
    ref_s = torch.zeros(ns, dtype=torch.float64, device="cuda")
    ref_a = torch.zeros(na, dtype=torch.float64, device="cuda")
    ctx.adjoint_sigma(prob, pts, 16, gu, ref_s, 1e-4, sb, seed=5)
    ctx.adjoint_alpha(prob, pts, 16, gu, ref_a, 1e-4, sb, seed=5)
    gs, ga = ctx.adjoint(prob, pts, 16, 1e-4, sb, gu, sigma_nodes=ns, alpha_nodes=na, seed=5)
    scale_s = float(ref_s.abs().max())
    scale_a = float(ref_a.abs().max())
    # FP32 walks: the replays' atomics add in a different order, so compare to rounding
    assert torch.allclose(gs.double(), ref_s, rtol=1e-5, atol=1e-6 * scale_s)
    assert torch.allclose(ga.double(), ref_a, rtol=1e-5, atol=1e-6 * scale_a)
    only_s, none_a = ctx.adjoint(prob, pts, 16, 1e-4, sb, gu, sigma_nodes=ns, seed=5)
    assert none_a is None and torch.allclose(only_s, gs, rtol=1e-5, atol=1e-6 * scale_s)


def test_open_mesh_is_rejected(wos, ctx):
    verts, tris = W.displaced_icosphere(2, 0.1, 3)
    v = torch.from_numpy(verts).cuda()
    t = torch.from_numpy(np.ascontiguousarray(tris[1:])).cuda()  # one face removed
    with pytest.raises(wos.WosError) as e:
        ctx.domain_mesh(v, t)
    assert e.value.code == wos.WOS_EINVAL
    flipped = tris.copy()
    flipped[0] = flipped[0][::-1]  # one face wound the other way
    with pytest.raises(wos.WosError):
        ctx.domain_mesh(v, torch.from_numpy(np.ascontiguousarray(flipped)).cuda())
    ctx.domain_mesh(v, torch.from_numpy(tris).cuda()).close()
