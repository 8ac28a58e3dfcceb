"""PyTorch autograd over the walk-on-spheres solve, for inverse problems.

`SigmaSolve.apply(sigma, ctx, prob, pts, walks, eps, sigma_bar, seed)` returns the
per-point estimates of wos_solve; its backward calls wos_adjoint_sigma, which
replays the same walks (same seed and walk ids) and returns the exact gradient of
those estimates with respect to the node values of the multilinear sigma grid
(given sigma_bar the walk paths do not depend on sigma, Sec. 5.1).  `sigma` must
be the device tensor the problem's sigma grid reads (the library keeps a pointer
to it), so updating it in place changes the next solve.  `CoefficientSolve` does the
same for sigma and the cubic B-spline alpha grid together.
"""
from __future__ import annotations

import torch


class SigmaSolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, sigma, ctx, prob, pts, walks, eps, sigma_bar, seed, precision="fp32"):
        if sigma.data_ptr() != prob.sigma_data_ptr():
            raise ValueError("sigma must be the tensor the problem's sigma grid was created from")
        acc, _ = ctx.solve(prob, pts, walks, eps, sigma_bar, seed=seed, precision=precision)
        mean, _, _ = ctx.finalize(acc)
        fctx.save_for_backward(pts)
        fctx.args = (ctx, prob, walks, eps, sigma_bar, seed, precision, sigma.shape)
        return mean

    @staticmethod
    def backward(fctx, grad_mean):
        (pts,) = fctx.saved_tensors
        ctx, prob, walks, eps, sigma_bar, seed, precision, shape = fctx.args
        grad = torch.zeros(shape, dtype=torch.float64, device=pts.device)
        ctx.adjoint_sigma(prob, pts, walks, grad_mean.contiguous().to(torch.float64), grad.view(-1), eps, sigma_bar,
                          seed=seed, precision=precision)
        return grad.to(torch.float32), None, None, None, None, None, None, None, None


class CoefficientSolve(torch.autograd.Function):
    """`CoefficientSolve.apply(sigma, alpha, ctx, prob, pts, walks, eps, sigma_bar, seed)`:
    the per-point estimates, differentiable with respect to both the multilinear sigma
    grid and the cubic B-spline alpha grid the problem reads (wos_adjoint_sigma and
    wos_adjoint_alpha replay the same walks).  Either input may be None (no gradient)."""

    @staticmethod
    def forward(fctx, sigma, alpha, ctx, prob, pts, walks, eps, sigma_bar, seed, precision="fp32"):
        if sigma is not None and sigma.data_ptr() != prob.sigma_data_ptr():
            raise ValueError("sigma must be the tensor the problem's sigma grid was created from")
        if alpha is not None and alpha.data_ptr() != prob.alpha_data_ptr():
            raise ValueError("alpha must be the tensor the problem's alpha grid was created from")
        acc, _ = ctx.solve(prob, pts, walks, eps, sigma_bar, seed=seed, precision=precision)
        mean, _, _ = ctx.finalize(acc)
        fctx.save_for_backward(pts)
        fctx.args = (ctx, prob, walks, eps, sigma_bar, seed, precision,
                     None if sigma is None else sigma.shape, None if alpha is None else alpha.shape)
        return mean

    @staticmethod
    def backward(fctx, grad_mean):
        (pts,) = fctx.saved_tensors
        ctx, prob, walks, eps, sigma_bar, seed, precision, sshape, ashape = fctx.args
        gu = grad_mean.contiguous().to(torch.float64)
        gs = ga = None
        if sshape is not None and fctx.needs_input_grad[0]:
            g = torch.zeros(sshape, dtype=torch.float64, device=pts.device)
            ctx.adjoint_sigma(prob, pts, walks, gu, g.view(-1), eps, sigma_bar, seed=seed, precision=precision)
            gs = g.to(torch.float32)
        if ashape is not None and fctx.needs_input_grad[1]:
            g = torch.zeros(ashape, dtype=torch.float64, device=pts.device)
            ctx.adjoint_alpha(prob, pts, walks, gu, g.view(-1), eps, sigma_bar, seed=seed, precision=precision)
            ga = g.to(torch.float32)
        return gs, ga, None, None, None, None, None, None, None, None
