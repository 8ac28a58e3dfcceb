"""GPU parity of the extra-drift walks (a drift that is not alpha times a gradient; the
drift term moved onto the Green's function by parts on each ball) with the oracle.

* FP64 replay: per walk equal to the oracle's on the same Philox streams (>= 99%).
* FP32: the manufactured solutions within 4 standard errors, including the cube
  workload with its literal omega = (sin 2 pi y, cos 2 pi z, 0.5).
* Entry points without the drift term refuse such problems.
"""
import numpy as np
import pytest

import workloads as W
from tests.stats_util import four_se_rule
from tests.test_oracle_drift import CASES

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


@pytest.mark.parametrize("name", list(CASES))
def test_drift_fp64_replay_per_walk(orc, ctx, name):
    mk, exact, ptsf, _ = CASES[name]
    desc = mk()
    pts = ptsf()
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc)[0]
    uh, st, _ = ctx.walk_estimates(prob, dev(pts), 16, 1e-4, sb, seed=4, precision="fp64")
    uo, so = orc.walks(desc, pts, 16, seed=4, eps=1e-4, sigma_bar=sb)
    ok = np.abs(uh.cpu().numpy() - uo) <= 1e-9 * np.maximum(1.0, np.abs(uo))
    assert ok.mean() >= 0.99 and (st.cpu().numpy() == so).mean() >= 0.99, ok.mean()


@pytest.mark.parametrize("name", list(CASES))
def test_drift_fp32_exact_solution(orc, ctx, name):
    mk, exact, ptsf, _ = CASES[name]
    desc = mk()
    pts = ptsf()
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc)[0]
    # the GPU's own sigma_bar prepass includes the drift terms too
    sbg = ctx.sigma_bar(prob, 64 if desc["dim"] == 3 else 256)[0]
    assert abs(sbg - sb) <= 0.05 * sb
    acc, stats = ctx.solve(prob, dev(pts), 1 << 15, 1e-4, sb, seed=6)
    m, v, se = (t.cpu().numpy() for t in ctx.finalize(acc))
    ok, nout, mz = four_se_rule((m - exact(pts.astype(np.float64))) / se)
    assert ok, (name, nout, mz)


def test_drift_full_cube_literal_rms(orc, ctx):
    """Config 2 as stated (non-conservative omega): 64^3 points x 1024 walks, sampled points
    against the exact solution."""
    desc = W.cube3d_literal_problem()
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc)[0]
    pts = W.cell_centres(3, 64)
    acc, stats = ctx.solve(prob, dev(pts), 1024, 1e-4, sb, seed=0)
    m, v, se = (t.cpu().numpy() for t in ctx.finalize(acc))
    idx = W.seeded_subset(64 ** 3, 4096, 3)
    z = (m[idx] - W.cube3d_exact(*pts[:, idx].astype(np.float64))) / se[idx]
    ok, nout, mz = four_se_rule(z)
    assert ok, (nout, mz)
    # FP32 uniforms can equal the mixture's split point: every walk must stay finite
    s = [int(x) for x in stats.cpu().tolist()]
    assert s[1] == 64 ** 3 * 1024 and s[2] == 0 and s[3] == 0, s
    assert np.all(np.isfinite(m))


def test_drift_refused_where_the_term_is_missing(orc, ctx, wos):
    desc = W.cube3d_literal_problem()
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc)[0]
    pts = dev(W.cell_centres(3, 4))
    for call in (lambda: ctx.solve_grad(prob, pts, 4, 1e-4, sb), lambda: ctx.solve_nf(prob, pts, 4, 1e-4, sb),
                 lambda: ctx.solve(prob, pts, 4, 1e-4, sb, window=(0.5, 1.5, 4))):
        with pytest.raises(wos.WosError) as e:
            call()
        assert e.value.code == wos.WOS_EUNSUPPORTED
