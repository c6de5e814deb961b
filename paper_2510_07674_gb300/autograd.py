"""Differentiable SPaSM costs for PyTorch (torch.autograd.Function around the CUDA kernels).

``traj_cost(problem, q, lam, mu)`` is the stage-2 augmented-Lagrangian objective of each
trajectory particle (Sec. III-B; cost terms of the appendix) and ``place_cost(problem, x,
quadratic)`` the stage-1 tower placement cost (appendix, Alg. 1's linear / quadratic forms).
The forward pass runs the evaluation kernel without its backward part; the backward pass
runs the kernel again with the analytic backward, recomputing the forward kinematics
instead of storing transforms, and scales the per-particle gradient by the incoming
gradient.  Inputs are CUDA float32 tensors; no computation happens in Python.
"""
from __future__ import annotations

import torch

from . import spasm as S


def _pad8(q: torch.Tensor, C: int) -> torch.Tensor:
    if q.dim() != 3 or q.shape[1] != C or q.shape[2] not in (7, 8):
        raise ValueError(f"q must be (n, {C}, 7|8)")
    if q.shape[2] == 8:
        return q.detach().contiguous().float()
    out = torch.zeros(q.shape[0], C, 8, device=q.device, dtype=torch.float32)
    out[:, :, :7] = q.detach()
    return out


class TrajCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, problem, lam, mu):
        qq = _pad8(q, problem.C)
        n = qq.shape[0]
        L = torch.empty(n, device=q.device, dtype=torch.float32)
        lam_c = None if lam is None else lam.detach().contiguous().float()
        mu_c = None if mu is None else mu.detach().contiguous().float()
        S.spasm_traj_eval(problem, n, qq, lam_c, mu_c, L, None)
        ctx.problem = problem
        ctx.width = q.shape[2]
        ctx.save_for_backward(qq, *(t for t in (lam_c, mu_c) if t is not None))
        ctx.has_lam, ctx.has_mu = lam_c is not None, mu_c is not None
        return L

    @staticmethod
    def backward(ctx, gL):
        saved = list(ctx.saved_tensors)
        qq = saved.pop(0)
        lam_c = saved.pop(0) if ctx.has_lam else None
        mu_c = saved.pop(0) if ctx.has_mu else None
        n = qq.shape[0]
        L = torch.empty(n, device=qq.device, dtype=torch.float32)
        grad = torch.empty_like(qq)
        S.spasm_traj_eval(ctx.problem, n, qq, lam_c, mu_c, L, grad)
        g = grad[:, :, : ctx.width] * gL.to(grad.dtype)[:, None, None]
        return g, None, None, None


class PlaceCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, problem, quadratic):
        xx = x.detach().contiguous().float()   # (4B, n) structure of arrays
        n = xx.shape[1]
        cost = torch.empty(n, device=x.device, dtype=torch.float32)
        S.spasm_place_eval(problem, n, xx, int(quadratic), cost, None)
        ctx.problem, ctx.quadratic = problem, int(quadratic)
        ctx.save_for_backward(xx)
        return cost

    @staticmethod
    def backward(ctx, gc):
        (xx,) = ctx.saved_tensors
        n = xx.shape[1]
        cost = torch.empty(n, device=xx.device, dtype=torch.float32)
        grad = torch.empty_like(xx)
        S.spasm_place_eval(ctx.problem, n, xx, ctx.quadratic, cost, grad)
        return grad * gc.to(grad.dtype)[None, :], None, None


def traj_cost(problem, q, lam=None, mu=None):
    """Per-particle stage-2 objective L(q) (n,), differentiable w.r.t. q (n, C, 7|8)."""
    return TrajCost.apply(q, problem, lam, mu)


def place_cost(problem, x, quadratic: bool = False):
    """Per-particle stage-1 placement cost (n,), differentiable w.r.t. x (4B, n)."""
    return PlaceCost.apply(x, problem, quadratic)
