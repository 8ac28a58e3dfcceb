"""The allocation-free solve (wos_solve_noalloc) against the regular wos_solve.

wos_solve_noalloc is for callers that cannot allocate device memory (allocator
hooks, plugins whose host program owns all allocations, code that must not
synchronise the device as cudaFree does).  It keeps its scratch in a static
device array, so these checks call it through the C interface and compare its
accumulators with those of the regular entry point on the same inputs, on two
calls in a row (the static scratch keeps the previous call's contents):

* FP64 walks run identical arithmetic on identical random streams: the sums
  agree to summation-order rounding (1e-9 relative), counts exactly;
* FP32 walks start Newton differently, so the means agree within 4 combined
  standard errors;
* per-point walk counts up to the static limit, the limit itself, and a call
  that fills the static prefix-sum buffer exactly;
* a call on a stream other than the current one.
"""
import ctypes as C

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
    lib = m.load()
    lib.wos_solve_noalloc.argtypes = [C.POINTER(m.ProblemDesc), C.c_void_p, C.c_int64, C.c_void_p, C.c_int32,
                                      C.POINTER(m.Params), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]
    return m


FIELD_KINDS = {"zero": 0, "const": 1, "sst": 2, "manufactured": 3, "grid_linear": 4, "grid_bspline": 5}
DOM_KINDS = {"box": 0, "ball": 1, "annulus": 2, "rounded_box": 3}


def pack(wos, desc, keep):
    """A workloads problem dict as the C struct wos_problem_desc (grids uploaded to cuda:0)."""
    D = wos.ProblemDesc()
    D.dim = desc["dim"]
    D.domain.kind = DOM_KINDS[desc["domain"]["kind"]]
    for i, v in enumerate(desc["domain"]["p"]):
        D.domain.p[i] = v
    for name in ("alpha", "phi", "sigma", "f", "g", "um"):
        fd = desc[name]
        F = getattr(D, name)
        F.kind = FIELD_KINDS[fd["kind"]]
        F.value = fd.get("value", 0.0)
        if fd["kind"] == "sst":
            terms = (wos.Term * max(1, len(fd["terms"])))()
            for i, t in enumerate(fd["terms"]):
                terms[i].c = t["c"]
                for d, (ty, k, ph) in enumerate(t["atoms"]):
                    terms[i].type[d], terms[i].k[d], terms[i].phi[d] = ty, k, ph
            keep.append(terms)
            F.nterms = len(fd["terms"])
            F.terms = C.cast(terms, C.POINTER(wos.Term))
        if fd["kind"].startswith("grid"):
            data = torch.from_numpy(np.ascontiguousarray(fd["data"], dtype=np.float32)).cuda()
            keep.append(data)
            for d in range(3):
                F.res[d] = fd["res"][d] if d < len(fd["res"]) else 1
                F.lo[d] = fd["lo"][d] if d < len(fd["lo"]) else 0.0
                F.hi[d] = fd["hi"][d] if d < len(fd["hi"]) else 0.0
            F.data = data.data_ptr()
    return D


def noalloc(wos, D, pts, walks, prm, acc, stats=None, stream=None):
    st = torch.cuda.current_stream() if stream is None else stream
    if isinstance(walks, int):
        wp, wu = None, walks
    else:
        wp, wu = C.c_void_p(walks.data_ptr()), 0
    rc = wos.load().wos_solve_noalloc(C.byref(D), C.c_void_p(pts.data_ptr()), pts.shape[1], wp, wu, C.byref(prm),
                                      C.c_void_p(acc[0].data_ptr()), C.c_void_p(acc[1].data_ptr()),
                                      C.c_void_p(acc[2].data_ptr()),
                                      None if stats is None else C.c_void_p(stats.data_ptr()),
                                      C.c_void_p(st.cuda_stream))
    return rc


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("name", ["cube3d", "noise_annulus"])
def test_fp64_matches_regular_solve_two_calls(wos, orc, name):
    desc = W.cube3d_problem() if name == "cube3d" else W.noise_annulus_problem()
    eps = 1e-4 if name == "cube3d" else 1e-3
    pts = W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 200, 31)] if name == "cube3d" else \
        np.array([[0.5, -0.6, 0.0, 0.7], [0.2, 0.3, -0.8, -0.5]], dtype=np.float32)
    sb = orc.sigma_bar(desc, 64 if desc["dim"] == 3 else 128)[0]
    ctx = wos.Context(0)
    prob = ctx.problem(desc)
    keep = []
    D = pack(wos, desc, keep)
    p = dev(pts)
    ref = ctx.new_accum(p.shape[1])
    got = ctx.new_accum(p.shape[1])
    stats = ctx.new_stats()
    for call, offset in enumerate((0, 64)):
        ctx.solve(prob, p, 64, eps, sb, seed=21, walk_offset=offset, precision="fp64", accum=ref)
        prm = wos.params(eps, sb, seed=21, walk_offset=offset, precision="fp64")
        assert noalloc(wos, D, p, 64, prm, got, stats) == wos.WOS_OK
        torch.cuda.synchronize()
        assert torch.equal(ref[2], got[2]), call
        assert torch.allclose(ref[0], got[0], rtol=1e-9, atol=1e-12), call
        assert torch.allclose(ref[1], got[1], rtol=1e-9, atol=1e-12), call
    s = [int(v) for v in stats.cpu().tolist()]
    assert s[1] == 2 * 64 * p.shape[1] and s[2] == 0 and s[3] == 0


def test_fp32_statistics_match_regular_solve(wos, orc):
    desc = W.square2d_problem()
    sb = orc.sigma_bar(desc)[0]
    ctx = wos.Context(0)
    prob = ctx.problem(desc)
    keep = []
    D = pack(wos, desc, keep)
    p = dev(W.cell_centres(2, 32))
    for call in range(2):
        ref, _ = ctx.solve(prob, p, 512, 1e-3, sb, seed=40 + call)
        got = ctx.new_accum(p.shape[1])
        assert noalloc(wos, D, p, 512, wos.params(1e-3, sb, seed=40 + call), got) == wos.WOS_OK
        m1, _, se1 = (t.cpu().numpy() for t in ctx.finalize(ref))
        m2, _, se2 = (t.cpu().numpy() for t in ctx.finalize(got))
        assert torch.equal(ref[2], got[2])
        ok, nout, mz = four_se_rule(combined_z(m1, se1, m2, se2))
        assert ok, (call, nout, mz)


def test_per_point_walks_and_the_static_limit(wos, orc):
    desc = W.cube3d_problem()
    sb = orc.sigma_bar(desc, 64)[0]
    ctx = wos.Context(0)
    prob = ctx.problem(desc)
    keep = []
    D = pack(wos, desc, keep)
    pts = W.uniform_in_box(3, 3000, 0.02, 0.98, 32)
    walks = torch.from_numpy(np.random.default_rng(3).integers(0, 40, size=3000).astype(np.int32)).cuda()
    p = dev(pts)
    for call in range(2):
        ref, _ = ctx.solve(prob, p, walks, 1e-4, sb, seed=50 + call, precision="fp64")
        got = ctx.new_accum(p.shape[1])
        prm = wos.params(1e-4, sb, seed=50 + call, precision="fp64")
        assert noalloc(wos, D, p, walks, prm, got) == wos.WOS_OK
        torch.cuda.synchronize()
        assert torch.equal(ref[2], got[2]) and torch.equal(got[2].cpu().to(torch.int32), walks.cpu())
        assert torch.allclose(ref[0], got[0], rtol=1e-9, atol=1e-12)
    # beyond the static prefix-sum capacity the call is rejected, uniform counts are not limited
    big = torch.zeros((3, 65537), dtype=torch.float32, device="cuda") + 0.5
    bw = torch.ones(65537, dtype=torch.int32, device="cuda")
    acc = ctx.new_accum(65537)
    assert noalloc(wos, D, big, bw, wos.params(1e-4, sb), acc) == wos.WOS_EINVAL
    assert noalloc(wos, D, big, 1, wos.params(1e-4, sb), acc) == wos.WOS_OK
    torch.cuda.synchronize()
    assert int(acc[2].sum()) == 65537
    # invalid descriptions and parameters are rejected before any work
    bad = W.cube3d_problem()
    bad["alpha"] = W.const(0.0)
    Db = pack(wos, bad, keep)
    assert noalloc(wos, Db, p, 4, wos.params(1e-4, sb), ctx.new_accum(3000)) == wos.WOS_EINVAL
    assert noalloc(wos, D, p, 4, wos.params(0.0, sb), ctx.new_accum(3000)) == wos.WOS_EINVAL


def test_full_prefix_buffer_and_a_side_stream(wos, orc):
    """npts equal to the static limit fills the prefix-sum buffer to its last entry."""
    desc = W.cube3d_problem()
    sb = orc.sigma_bar(desc, 64)[0]
    ctx = wos.Context(0)
    prob = ctx.problem(desc)
    keep = []
    D = pack(wos, desc, keep)
    n = 65536  # WOS_NOALLOC_MAX_VAR_POINTS
    pts = W.uniform_in_box(3, n, 0.02, 0.98, 33)
    walks = torch.from_numpy(np.random.default_rng(4).integers(0, 3, size=n).astype(np.int32)).cuda()
    p = dev(pts)
    ref, _ = ctx.solve(prob, p, walks, 1e-4, sb, seed=61, precision="fp64")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        got = ctx.new_accum(n)
    prm = wos.params(1e-4, sb, seed=61, precision="fp64")
    for call in range(2):
        with torch.cuda.stream(side):
            for t in got:
                t.zero_()
        assert noalloc(wos, D, p, walks, prm, got, stream=side) == wos.WOS_OK
        side.synchronize()
        assert torch.equal(ref[2], got[2]), call
        assert torch.equal(got[2].cpu().to(torch.int32), walks.cpu()), call
        assert torch.allclose(ref[0], got[0], rtol=1e-9, atol=1e-12), call
        assert torch.allclose(ref[1], got[1], rtol=1e-9, atol=1e-12), call
