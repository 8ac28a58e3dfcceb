"""The progressive slice view (Sec. 7.2): slice points, one walk per point per frame,
and the sphere-traced image of the domain cut by the slice plane.

* Geometry: for a ball cut by a plane through its centre, every pixel's ray depth
  equals the analytic intersection with the remaining half (or a miss).
* Values: pixels on the slice show sum / count of their slice cell.
* Progressive accumulation: F frames of one walk each equal one solve of F walks
  (same walk ids); editing the problem discards the accumulated walks.
"""
import math

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


def test_ball_cut_by_plane_depth_and_values(wos, ctx):
    desc = W.laplace_ball_problem()
    prob = ctx.problem(desc)
    v = wos.view([-1.2, -1.2, 0.0], [2.4, 0, 0], [0, 2.4, 0], 64, 64, 96, 80, (-2.0, 2.0), eye=(0.3, -0.2, 4.0),
                 look=(0, 0, 0), up=(0, 1, 0), fov_y_deg=35.0)
    pts = ctx.slice_points(prob, v)
    acc, _ = ctx.solve(prob, pts, 64, 1e-4, 1e-3, seed=1)
    img, val, dep = ctx.render_slice(prob, v, acc, with_value=True, with_depth=True)
    img, val, dep = img.cpu().numpy(), val.cpu().numpy(), dep.cpu().numpy()
    assert img.shape == (80, 96, 4) and np.all(img[:, :, 3] == 255)
    # the camera basis of the view (pinhole)
    eye = np.array([0.3, -0.2, 4.0])
    fwd = -eye / np.linalg.norm(eye)
    right = np.cross(fwd, [0, 1, 0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    th = math.tan(math.radians(35.0) / 2)
    mean = (acc[0] / acc[2].clamp(min=1)).cpu().numpy()
    checked = 0
    for py in range(80):
        for px in range(96):
            sx = ((px + 0.5) / 96 * 2 - 1) * th * 96 / 80
            sy = (1 - (py + 0.5) / 80 * 2) * th
            d = fwd + sx * right + sy * up
            d /= np.linalg.norm(d)
            t = -eye[2] / d[2]  # z = 0
            q = eye + t * d
            rq = math.hypot(q[0], q[1])
            if abs(rq - 1.0) < 2e-2:
                continue  # rim pixels: grazing rays
            checked += 1
            if rq < 1.0:
                assert abs(dep[py, px] - t) <= 1e-4 * t, (px, py, dep[py, px], t)
                a, b = (q[0] + 1.2) / 2.4, (q[1] + 1.2) / 2.4
                cell = min(int(b * 64), 63) * 64 + min(int(a * 64), 63)
                assert abs(val[py, px] - mean[cell]) <= 1e-5 * max(1.0, abs(mean[cell]))
            else:
                # the ray passes the plane outside the disk and diverges below it: a miss
                assert np.isinf(dep[py, px]) and np.isnan(val[py, px])
    assert checked > 6000


def test_progressive_frames_equal_one_solve_and_edit_resets(wos, ctx, orc):
    desc = W.csg_laplace_problem(2)
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc)[0]
    v = wos.view([-1.2, -1.0], [2.8, 0], [0, 2.0], 48, 32, 140, 100, (-2.0, 4.0))
    sv = wos.SliceView(ctx, prob, v, 1e-4, sb, seed=3)
    for _ in range(8):
        img = sv.frame(1)
    assert img.shape == (100, 140, 4)
    acc, _ = ctx.solve(prob, sv.pts, 8, 1e-4, sb, seed=3)
    assert torch.equal(sv.accum[2], acc[2])
    # the same walks; per-lane partial sums are formed in FP32, so the order of the sums differs
    assert torch.allclose(sv.accum[0], acc[0], rtol=1e-5, atol=1e-6)
    # slice points outside the CSG domain end at once (and are counted as such)
    st = wos.stats_dict(sv.stats)
    assert 0 < st["outside"] < st["walks"] and st["walks"] == 8 * 48 * 32
    # the 2D image shows the slice cell means inside the domain
    img, val, _ = ctx.render_slice(prob, v, sv.accum, with_value=True)
    val = val.cpu().numpy()
    mean = (sv.accum[0] / sv.accum[2].clamp(min=1)).cpu().numpy()
    shown = np.isfinite(val)
    assert shown.mean() > 0.3
    ys, xs = np.nonzero(shown)
    for py, px in list(zip(ys, xs))[::97]:
        a, b = (px + 0.5) / 140, 1 - (py + 0.5) / 100
        cell = min(int(b * 32), 31) * 48 + min(int(a * 48), 47)
        assert abs(val[py, px] - mean[cell]) <= 1e-5 * max(1.0, abs(mean[cell]))
    sv.edit(ctx.problem(W.csg_laplace_problem(2)))
    assert int(sv.accum[2].sum()) == 0 and sv.frames == 0
    sv.frame(2, render=False)
    assert int(sv.accum[2].max()) == 2


def test_csg_scene_render_runs(wos, ctx, orc):
    desc = W.csg_variable_problem()
    prob = ctx.problem(desc)
    sb = orc.sigma_bar(desc)[0]
    v = wos.view([-1.3, -1.3, 0.05], [2.6, 0, 0], [0, 2.6, 0], 128, 128, 160, 120, (-3.0, 3.0),
                 eye=(2.5, 2.0, 3.5), look=(0, 0, 0))
    sv = wos.SliceView(ctx, prob, v, 1e-4, sb)
    for _ in range(4):
        img = sv.frame(1)
    img, val, dep = ctx.render_slice(prob, v, sv.accum, with_value=True, with_depth=True)
    dep = dep.cpu().numpy()
    assert np.isfinite(dep).mean() > 0.1 and np.isfinite(val.cpu().numpy()).sum() > 100
    with pytest.raises(wos.WosError):
        ctx.render_slice(prob, wos.view([0, 0, 0], [0, 0, 0], [0, 1, 0], 4, 4, 8, 8, (0, 1)), ctx.new_accum(16))
