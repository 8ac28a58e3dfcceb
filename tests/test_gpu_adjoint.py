"""The path-replay gradients (wos_adjoint_sigma, wos_adjoint_alpha) against the
oracle's central finite differences with common random numbers: the oracle reruns
the same walks (same seed and walk ids) with one sigma or alpha node moved by +-h;
given sigma_bar the paths do not move, so the difference quotient has no Monte
Carlo noise."""
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
def setup(wos, orc):
    sig = W.inverse_sigma_grid()
    desc = W.inverse_problem(sig)
    sb = orc.sigma_bar(desc, 48)[0]
    pts = W.inverse_sensors(12, seed=5)
    grad_u = np.random.default_rng(6).normal(size=pts.shape[1])
    return sig, desc, sb, pts, grad_u


def oracle_fd(orc, sig, pts, grad_u, node, walks, seed, sb, h):
    """sum_p grad_u[p] d mean_p / d sigma_node by central differences on the same walks."""
    vals, nodes = [], []
    for s in (+1, -1):
        g = sig.copy().reshape(-1)
        g[node] += s * h
        nodes.append(float(g[node]))  # the float32 grid rounds the step: divide by what was applied
        desc = W.inverse_problem(g.reshape(sig.shape))
        uh, _ = orc.walks(desc, pts, walks, seed=seed, eps=1e-4, sigma_bar=sb)
        vals.append((grad_u * uh.mean(axis=1)).sum())
    return (vals[0] - vals[1]) / (nodes[0] - nodes[1])


def pick_nodes(sig, pts, k=6):
    """Grid nodes next to the first sensors (their gradients are not zero)."""
    n = sig.shape[0]
    out = []
    for i in range(k):
        x = pts[:, i % pts.shape[1]]
        ijk = np.clip(np.floor(x * (n - 1)).astype(int), 0, n - 2)
        out.append(int(ijk[0] + n * (ijk[1] + n * ijk[2])))
    return out


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-6), ("fp32", 5e-2)])
def test_adjoint_matches_crn_central_differences(wos, orc, setup, precision, rtol):
    sig, desc, sb, pts, grad_u = setup
    ctx = wos.Context(0)
    sig_t = torch.from_numpy(sig).cuda()
    d = dict(desc)
    d["sigma"] = dict(desc["sigma"], data=sig_t)
    prob = ctx.problem(d)
    walks, seed = 32, 9
    grad = torch.zeros(sig.size, dtype=torch.float64, device="cuda")
    ctx.adjoint_sigma(prob, torch.from_numpy(pts).cuda(), walks, torch.from_numpy(grad_u).cuda(), grad, 1e-4, sb,
                      seed=seed, precision=precision)
    g = grad.cpu().numpy()
    assert np.isfinite(g).all() and np.abs(g).sum() > 0
    for node in pick_nodes(sig, pts):
        fd = oracle_fd(orc, sig, pts, grad_u, node, walks, seed, sb, h=1e-3)
        scale = max(abs(fd), 1e-3 * np.abs(g).max())
        assert abs(g[node] - fd) <= rtol * scale, (precision, node, g[node], fd)


def test_autograd_function_and_descent(wos, orc, setup):
    """loss.backward() through SigmaSolve equals the adjoint, and gradient steps on the
    sigma grid lower an L2 misfit to a target solved with the hidden sigma."""
    from paper_2201_13240_gb300.autograd import SigmaSolve
    sig_true, desc, sb, _, _ = setup
    ctx = wos.Context(0)
    pts = torch.from_numpy(W.inverse_sensors(256, seed=7)).cuda()
    t_true = torch.from_numpy(sig_true).cuda()
    dt = dict(desc)
    dt["sigma"] = dict(desc["sigma"], data=t_true)
    acc, _ = ctx.solve(ctx.problem(dt), pts, 4096, 1e-4, sb, seed=100)
    target = ctx.finalize(acc)[0]
    sigma = torch.full_like(t_true, 5.0).requires_grad_(True)
    d = dict(desc)
    d["sigma"] = dict(desc["sigma"], data=sigma.detach())
    prob = ctx.problem(d)
    losses = []
    for it in range(4):
        u = SigmaSolve.apply(sigma, ctx, prob, pts, 256, 1e-4, sb, 200 + it)
        loss = ((u - target) ** 2).sum()
        sigma.grad = None
        loss.backward()
        assert sigma.grad is not None and torch.isfinite(sigma.grad).all()
        if it == 0:
            ref = torch.zeros(sigma.numel(), dtype=torch.float64, device="cuda")
            ctx.adjoint_sigma(prob, pts, 256, (2 * (u - target)).detach(), ref, 1e-4, sb, seed=200)
            assert torch.allclose(sigma.grad.reshape(-1).double(), ref, rtol=1e-5, atol=1e-9)
        losses.append(float(loss.detach()))
        with torch.no_grad():
            sigma -= 0.5 * sigma.grad / sigma.grad.abs().max()
            sigma.clamp_(0.0, 20.0)
    assert losses[-1] < losses[0]


def oracle_fd_alpha(orc, sig, alpha, pts, grad_u, node, walks, seed, sb, h):
    """sum_p grad_u[p] d mean_p / d alpha_node (B-spline control value) on the same walks."""
    vals, nodes = [], []
    for s in (+1, -1):
        a = alpha.copy().reshape(-1)
        a[node] += s * h
        nodes.append(float(a[node]))
        desc = W.inverse_problem(sig, a.reshape(alpha.shape))
        uh, _ = orc.walks(desc, pts, walks, seed=seed, eps=1e-4, sigma_bar=sb)
        vals.append((grad_u * uh.mean(axis=1)).sum())
    return (vals[0] - vals[1]) / (nodes[0] - nodes[1])


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-6), ("fp32", 5e-2)])
def test_alpha_adjoint_matches_crn_central_differences(wos, orc, setup, precision, rtol):
    """The alpha-grid gradient (e^{-gamma(x0)}, f', the null weights through sigma', and
    e^{gamma(x_n)}) against central differences of the oracle on the same walks."""
    sig, desc, sb, pts, grad_u = setup
    alpha = W.inverse_alpha_grid()
    ctx = wos.Context(0)
    d = dict(desc)
    d["sigma"] = dict(desc["sigma"], data=torch.from_numpy(sig).cuda())
    d["alpha"] = dict(desc["alpha"], data=torch.from_numpy(alpha).cuda())
    prob = ctx.problem(d)
    walks, seed = 32, 11
    grad = torch.zeros(alpha.size, dtype=torch.float64, device="cuda")
    ctx.adjoint_alpha(prob, torch.from_numpy(pts).cuda(), walks, torch.from_numpy(grad_u).cuda(), grad, 1e-4, sb,
                      seed=seed, precision=precision)
    g = grad.cpu().numpy()
    assert np.isfinite(g).all() and np.abs(g).sum() > 0
    n = alpha.shape[0]
    for i in range(6):
        x = pts[:, i]
        ijk = np.clip(np.floor(x * (n - 1)).astype(int) + (i % 2), 0, n - 1)
        node = int(ijk[0] + n * (ijk[1] + n * ijk[2]))
        fd = oracle_fd_alpha(orc, sig, alpha, pts, grad_u, node, walks, seed, sb, h=1e-3)
        scale = max(abs(fd), 1e-3 * np.abs(g).max())
        assert abs(g[node] - fd) <= rtol * scale, (precision, node, g[node], fd)


def test_coefficient_solve_backward_matches_adjoints(wos, orc, setup):
    from paper_2201_13240_gb300.autograd import CoefficientSolve
    sig, desc, sb, _, _ = setup
    ctx = wos.Context(0)
    pts = torch.from_numpy(W.inverse_sensors(128, seed=8)).cuda()
    s_t = torch.from_numpy(sig).cuda().requires_grad_(True)
    a_t = torch.from_numpy(W.inverse_alpha_grid()).cuda().requires_grad_(True)
    d = dict(desc)
    d["sigma"] = dict(desc["sigma"], data=s_t.detach())
    d["alpha"] = dict(desc["alpha"], data=a_t.detach())
    prob = ctx.problem(d)
    u = CoefficientSolve.apply(s_t, a_t, ctx, prob, pts, 64, 1e-4, sb, 5)
    w = torch.linspace(-1, 1, u.numel(), device="cuda", dtype=torch.float64)
    (u * w).sum().backward()
    rs = torch.zeros(sig.size, dtype=torch.float64, device="cuda")
    ra = torch.zeros(a_t.numel(), dtype=torch.float64, device="cuda")
    ctx.adjoint_sigma(prob, pts, 64, w, rs, 1e-4, sb, seed=5)
    ctx.adjoint_alpha(prob, pts, 64, w, ra, 1e-4, sb, seed=5)
    # the FP32 replay sums in nondeterministic order (per-CTA FP32 partial sums for alpha)
    assert torch.allclose(s_t.grad.reshape(-1).double(), rs, rtol=1e-4, atol=1e-6 * float(rs.abs().max()))
    assert torch.allclose(a_t.grad.reshape(-1).double(), ra, rtol=1e-3, atol=1e-4 * float(ra.abs().max()))


def test_sigma_adjoint_matches_fd_grid_reference(wos, orc):
    """The path-replay gradient's expectation is the gradient of the PDE solution: against the
    discrete adjoint of a second-order finite-difference solve (62 intervals, aligned with the
    sigma grid's nodes; ~3% discretisation error at this size), at 2^16 walks per sensor."""
    from tests.fd_reference import fd_cube_sigma_gradient
    sig = W.inverse_sigma_grid()
    alpha = W.inverse_alpha_grid()
    desc = W.inverse_problem(sig)
    pts = W.inverse_sensors(64, seed=4)
    w = np.random.default_rng(0).normal(size=64)
    u_fd, g_fd = fd_cube_sigma_gradient(alpha, sig, lambda x, y, z: np.ones_like(x),
                                        lambda x, y, z: 1 + x * y + z, 62, pts.astype(np.float64), w)
    ctx = wos.Context(0)
    d = dict(desc)
    d["sigma"] = dict(desc["sigma"], data=torch.from_numpy(sig).cuda())
    prob = ctx.problem(d)
    sb = orc.sigma_bar(desc, 48)[0]
    p = torch.from_numpy(pts).cuda()
    acc, _ = ctx.solve(prob, p, 1 << 16, 1e-4, sb, seed=21)
    m, v, se = (t.cpu().numpy() for t in ctx.finalize(acc))
    assert np.all(np.abs(m - u_fd) <= 4 * se + 2e-3)
    gs = []
    for seed in (21, 22):  # two independent halves give the Monte Carlo noise of their mean
        grad = torch.zeros(sig.size, dtype=torch.float64, device="cuda")
        ctx.adjoint_sigma(prob, p, 1 << 17, torch.from_numpy(w).cuda(), grad, 1e-4, sb, seed=seed)
        gs.append(grad.cpu().numpy())
    g = 0.5 * (gs[0] + gs[1])
    noise = 0.5 * np.linalg.norm(gs[0] - gs[1])
    err = np.linalg.norm(g - g_fd)
    # Monte Carlo noise (2 sigma) plus the reference's discretisation error (5% allowance)
    assert err <= 2.0 * noise + 0.05 * np.linalg.norm(g_fd), (err, noise, np.linalg.norm(g_fd))
    assert err <= 0.15 * np.linalg.norm(g_fd)


def test_specialised_adjoints_equal_the_generic_ones(wos, orc, setup):
    """WOS_SPEC_ADJOINT: the replay kernels compiled for the problem's fields give the
    generic kernels' gradients (FP64 to summation-order rounding; FP32 to its rounding) and,
    in FP64, the oracle's common-random-number central differences."""
    sig, desc, sb, pts, grad_u = setup
    ctx = wos.Context(0)
    d = dict(desc)
    d["sigma"] = dict(desc["sigma"], data=torch.from_numpy(sig).cuda())
    gen = ctx.problem(d)
    spec = ctx.problem(d, specialize=(("fp32", "fp64"), ("plain", "adjoint")))
    assert spec.specialized() & wos.WOS_SPEC_ADJOINT
    p = torch.from_numpy(pts).cuda()
    gu = torch.from_numpy(grad_u).cuda()
    na = W.inverse_alpha_grid().size
    for precision, rtol in (("fp64", 1e-10), ("fp32", 2e-4)):
        out = {}
        for name, prob in (("gen", gen), ("spec", spec)):
            gs = torch.zeros(sig.size, dtype=torch.float64, device="cuda")
            ga = torch.zeros(na, dtype=torch.float64, device="cuda")
            ctx.adjoint_sigma(prob, p, 32, gu, gs, 1e-4, sb, seed=9, precision=precision)
            ctx.adjoint_alpha(prob, p, 32, gu, ga, 1e-4, sb, seed=9, precision=precision)
            out[name] = (gs.cpu().numpy(), ga.cpu().numpy())
        for k in range(2):
            a, b = out["gen"][k], out["spec"][k]
            assert np.allclose(b, a, rtol=rtol, atol=rtol * np.abs(a).max()), (precision, k)
    gs = torch.zeros(sig.size, dtype=torch.float64, device="cuda")
    ctx.adjoint_sigma(spec, p, 32, gu, gs, 1e-4, sb, seed=9, precision="fp64")
    g = gs.cpu().numpy()
    for node in pick_nodes(sig, pts, k=3):
        fd = oracle_fd(orc, sig, pts, grad_u, node, 32, 9, sb, h=1e-3)
        assert g[node] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(g).max())


def test_full_size_adjoints_match_gpu_crn_differences(wos, orc):
    """The inverse workload at its full size (4096 sensors x 1024 walks, the benchmark's
    sensors, grad_u = 1): both replay gradients in FP64 at sampled grid nodes against central
    differences of FP64 forward solves on the same walks (common random numbers: given
    sigma_bar the paths do not move, so the quotient has no Monte Carlo noise)."""
    sig, alpha = W.inverse_sigma_grid(), W.inverse_alpha_grid()
    desc = W.inverse_problem(sig)
    sb = orc.sigma_bar(desc, 48)[0]
    ctx = wos.Context(0)
    pts = torch.from_numpy(W.inverse_sensors(4096)).cuda()
    walks, seed = 1024, 4
    gu = torch.ones(4096, dtype=torch.float64, device="cuda")

    def loss(sig_np, alpha_np):
        prob = ctx.problem(W.inverse_problem(sig_np, alpha_np))
        acc, _ = ctx.solve(prob, pts, walks, 1e-4, sb, seed=seed, precision="fp64")
        mean = ctx.finalize(acc)[0]
        prob.close()
        return float(mean.sum())

    prob = ctx.problem(desc)
    gs = torch.zeros(sig.size, dtype=torch.float64, device="cuda")
    ga = torch.zeros(alpha.size, dtype=torch.float64, device="cuda")
    ctx.adjoint_sigma(prob, pts, walks, gu, gs, 1e-4, sb, seed=seed, precision="fp64")
    ctx.adjoint_alpha(prob, pts, walks, gu, ga, 1e-4, sb, seed=seed, precision="fp64")
    gs, ga = gs.cpu().numpy(), ga.cpu().numpy()
    assert np.isfinite(gs).all() and np.isfinite(ga).all()
    for grid, g, which in ((sig, gs, "sigma"), (alpha, ga, "alpha")):
        # the nodes with the largest gradients, and one in the middle of the ranking
        order = np.argsort(-np.abs(g))
        for node in (int(order[0]), int(order[1]), int(order[len(order) // 4])):
            vals, steps = [], []
            for sgn in (+1, -1):
                m = grid.copy().reshape(-1)
                h = 1e-3 * max(abs(float(m[node])), 1.0)
                m[node] += sgn * h
                steps.append(float(m[node]))
                m = m.reshape(grid.shape)
                vals.append(loss(m, alpha) if which == "sigma" else loss(sig, m))
            fd = (vals[0] - vals[1]) / (steps[0] - steps[1])
            scale = max(abs(fd), 1e-3 * np.abs(g).max())
            assert abs(g[node] - fd) <= 1e-5 * scale, (which, node, g[node], fd)
