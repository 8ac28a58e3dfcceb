"""Batched solves: many independent 2D problems in one persistent launch.

* FP64: every sampled walk equals the oracle's walk of the same problem, point
  index (its index in the batch) and walk id;
* FP32: per-point agreement with the oracle within 4 combined standard errors;
* the launch replays inside a CUDA graph and gives the direct launch's counts and,
  in FP64, its sums.
"""
import numpy as np
import pytest

import workloads as W
from tests.stats_util import combined_z, four_se_rule

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
def setup(wos, orc):
    probs, pts, offs, walks = W.batch_problems(24, seed=11, max_points=48, min_points=4, min_walks=8, max_walks=64)
    sbs = np.array([orc.sigma_bar(p, 96)[0] for p in probs])
    ctx = wos.Context(0)
    hp = [ctx.problem(p) for p in probs]
    batch = ctx.batch(hp, offs, sbs)
    return ctx, probs, pts, offs, walks, sbs, batch


def prob_of(offs, i):
    return int(np.searchsorted(offs, i, side="right") - 1)


def test_fp64_walks_equal_oracle_walks(wos, orc, setup):
    ctx, probs, pts, offs, walks, sbs, batch = setup
    acc, st = ctx.solve_batch(batch, torch.from_numpy(pts).cuda(), 6, 1e-3, seed=13, precision="fp64")
    mean, var, se = (t.cpu().numpy() for t in ctx.finalize(acc))
    counts = acc[2].cpu().numpy()
    assert (counts == 6).all()
    rng = np.random.default_rng(0)
    packs = {}
    for i in rng.choice(pts.shape[1], size=40, replace=False):
        k = prob_of(offs, i)
        pk = packs.setdefault(k, orc.pack(probs[k]))
        u = [orc.walk(probs[k], pts[:, i].astype(np.float64), int(i), j, 13, 1e-3, sbs[k], packed=pk)[0]
             for j in range(6)]
        # the batch mean of the 6 walks equals the mean of the oracle's 6 walks
        assert mean[i] == pytest.approx(np.mean(u), rel=1e-9, abs=1e-9), (i, k)


def test_fp32_matches_oracle_statistics(wos, orc, setup):
    ctx, probs, pts, offs, walks, sbs, batch = setup
    acc, st = ctx.solve_batch(batch, torch.from_numpy(pts).cuda(), 512, 1e-3, seed=21)
    mean, var, se = (t.cpu().numpy() for t in ctx.finalize(acc))
    s = [int(v) for v in st.cpu().tolist()]
    assert s[1] == 512 * pts.shape[1] and s[2] == 0 and s[3] == 0
    zs = []
    for k in range(len(probs)):
        a, b = offs[k], offs[k + 1]
        oacc, _ = orc.solve(probs[k], pts[:, a:b], 512, seed=22, eps=1e-3, sigma_bar=sbs[k])
        om, ov, ose = orc.finalize(oacc)
        zs.append(combined_z(mean[a:b], se[a:b], om, ose))
    ok, nout, mz = four_se_rule(np.concatenate(zs))
    assert ok, (nout, mz)


def test_per_point_walks_and_graph_replay(wos, orc, setup):
    ctx, probs, pts, offs, walks, sbs, batch = setup
    p = torch.from_numpy(pts).cuda()
    w = torch.from_numpy(walks).cuda()
    ref, _ = ctx.solve_batch(batch, p, w, 1e-3, seed=31, precision="fp64")
    assert np.array_equal(ref[2].cpu().numpy(), walks)
    acc = ctx.new_accum(pts.shape[1])
    stats = ctx.new_stats()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):  # warm-up on the capture stream
        ctx.solve_batch(batch, p, w, 1e-3, seed=31, precision="fp64", accum=acc, stats=stats, stream=stream)
    torch.cuda.current_stream().wait_stream(stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        for t in acc:
            t.zero_()
        ctx.solve_batch(batch, p, w, 1e-3, seed=31, precision="fp64", accum=acc, stats=stats, stream=stream)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(acc[2], ref[2])
        assert torch.allclose(acc[0], ref[0], rtol=1e-9, atol=1e-12)
        assert torch.allclose(acc[1], ref[1], rtol=1e-9, atol=1e-12)


def test_schedules_change_the_lanes_not_the_walks(wos, setup):
    """Any schedule runs the same walks: FP64 sums equal the default schedule's to rounding,
    counts exactly; invalid schedules are refused."""
    ctx, probs, pts, offs, walks, sbs, batch = setup
    dpts = torch.from_numpy(pts).cuda()
    wt = torch.from_numpy(walks).cuda()
    batch.set_schedule()
    ref, _ = ctx.solve_batch(batch, dpts, wt, 1e-3, seed=5, precision="fp64")
    for sched in ({"chunk": 32}, {"chunk": 64, "blocks_per_sm": 1}, {"chunk": 2048, "regs_variant": 1},
                  {"chunk": 0, "blocks_per_sm": 3, "regs_variant": 1}):
        batch.set_schedule(**sched)
        assert {k: v for k, v in batch.schedule().items() if k in sched} == sched
        acc, st = ctx.solve_batch(batch, dpts, wt, 1e-3, seed=5, precision="fp64")
        assert torch.equal(acc[2], ref[2])
        assert torch.allclose(acc[0], ref[0], rtol=1e-12, atol=1e-12), sched
        acc32, _ = ctx.solve_batch(batch, dpts, wt, 1e-3, seed=5)
        assert torch.equal(acc32[2], ref[2])
    for bad in ({"chunk": 33}, {"chunk": 16}, {"blocks_per_sm": -1}, {"regs_variant": 2}, {"blocks_per_sm": 33}):
        with pytest.raises(wos.WosError):
            batch.set_schedule(**bad)
    batch.set_schedule()
    assert batch.schedule() == {"chunk": 0, "blocks_per_sm": 0, "regs_variant": 0}


def test_autotune_keeps_a_candidate_and_the_results(wos, setup):
    ctx, probs, pts, offs, walks, sbs, batch = setup
    dpts = torch.from_numpy(pts).cuda()
    wt = torch.from_numpy(walks).cuda()
    sched, best_ms, default_ms = ctx.batch_autotune(batch, dpts, wt, 1e-3, seed=1, trial_shift=2)
    assert sched["chunk"] in (0, 64, 128, 256, 512, 1024, 2048) and sched["regs_variant"] in (0, 1)
    assert 0 < best_ms <= default_ms
    assert batch.schedule() == sched
    acc, st = ctx.solve_batch(batch, dpts, wt, 1e-3, seed=9)
    assert torch.equal(acc[2].cpu(), torch.from_numpy(walks.astype(np.int64)))
    assert wos.stats_dict(st)["walks"] == int(walks.sum())
    with pytest.raises(wos.WosError):
        ctx.batch_autotune(batch, dpts, wt, 1e-3, trial_shift=17)
    batch.set_schedule()


def test_specialised_batch_runs_the_same_walks(wos, orc, setup):
    """wos_batch_specialize: the batched kernel with the shared fields compiled in gives the
    generic batched kernel's walks (FP64 sums to rounding, counts exact, both register caps)
    and the oracle's statistics in FP32."""
    ctx, probs, pts, offs, walks, sbs, batch = setup
    hp = [ctx.problem(p) for p in probs]
    spec = ctx.batch(hp, offs, sbs).specialize(("fp32", "fp64"))
    flags, uniform = spec.specialized()
    assert flags & wos.WOS_SPEC_FP32 and flags & wos.WOS_SPEC_FP64 and uniform == 0x3f
    p = torch.from_numpy(pts).cuda()
    w = torch.from_numpy(walks).cuda()
    ref, _ = ctx.solve_batch(batch, p, w, 1e-3, seed=41, precision="fp64")
    for regs in (0, 1):
        spec.set_schedule(regs_variant=regs)
        got, _ = ctx.solve_batch(spec, p, w, 1e-3, seed=41, precision="fp64")
        assert torch.equal(got[2], ref[2])
        assert torch.allclose(got[0], ref[0], rtol=1e-9, atol=1e-10)
    acc, st = ctx.solve_batch(spec, p, 512, 1e-3, seed=42)
    mean, var, se = (t.cpu().numpy() for t in ctx.finalize(acc))
    s = wos.stats_dict(st)
    assert s["walks"] == 512 * pts.shape[1] and s["capped"] == 0 and s["nonfinite"] == 0
    zs = []
    for k in range(len(probs)):
        a, b = offs[k], offs[k + 1]
        oacc, _ = orc.solve(probs[k], pts[:, a:b], 512, seed=43, eps=1e-3, sigma_bar=sbs[k])
        om, ov, ose = orc.finalize(oacc)
        zs.append(combined_z(mean[a:b], se[a:b], om, ose))
    ok, nout, mz = four_se_rule(np.concatenate(zs))
    assert ok, (nout, mz)


def test_full_size_batch_sampled_points(wos, orc):
    """The 4096-problem batch at its full size and in the benchmark's launch configuration
    (the batch kernel specialised to the shared fields, the autotuned schedule, per-point walk
    counts, one launch): 24 sampled points, each against the oracle's walks of its own problem
    at the same walk count, within 4 combined standard errors."""
    probs, pts, offs, walks = W.batch_problems(4096, seed=7)
    ctx = wos.Context(0)
    hp = [ctx.problem(p) for p in probs]
    sbs = [ctx.sigma_bar(h, 64)[0] for h in hp]
    batch = ctx.batch(hp, offs, sbs)
    batch.specialize(("fp32",))
    pts_t, wt = torch.from_numpy(pts).cuda(), torch.from_numpy(walks).cuda()
    ctx.batch_autotune(batch, pts_t, wt, 1e-3, seed=1, trial_shift=4)
    acc, st = ctx.solve_batch(batch, pts_t, wt, 1e-3, seed=0)
    mean, var, se = (t.cpu().numpy() for t in ctx.finalize(acc))
    s = wos.stats_dict(st)
    assert s["walks"] == int(walks.sum()) and s["capped"] == 0 and s["nonfinite"] == 0
    assert np.array_equal(acc[2].cpu().numpy(), walks.astype(np.int64))
    rng = np.random.default_rng(5)
    zs = []
    for i in rng.choice(pts.shape[1], size=24, replace=False):
        k = prob_of(offs, i)
        oacc, _ = orc.solve(probs[k], pts[:, i:i + 1], int(walks[i]), seed=3, eps=1e-3, sigma_bar=sbs[k])
        om, ov, ose = orc.finalize(oacc)
        zs.append(combined_z(mean[i:i + 1], se[i:i + 1], om, ose))
    ok, nout, mz = four_se_rule(np.concatenate(zs))
    assert ok, (nout, mz)
