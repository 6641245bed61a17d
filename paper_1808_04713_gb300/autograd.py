"""torch.autograd.Function for the plane-wave Helmholtz solve as a function of the element
permittivities.  Forward: set eps, factor, solve (all in libddh).  Backward: the transposed
adjoint system A^T lam = conj(G) is an ordinary solve on the same kernels (A is complex
symmetric), then the per-element gradient-accumulation kernel gives
dJ/deps_e = k^2 (h_e/2)^2 Re(lam_e^T M_e u_e).
"""
from __future__ import annotations

import torch


class PlaneWaveSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps: torch.Tensor, solver, thetas, tol: float = 1e-12, factor_opts: dict | None = None):
        solver.set_coefficients(solver_k(solver), eps.detach().cpu().double().numpy())
        solver.factor(**(factor_opts or {}))
        b = solver.rhs_planewave(thetas)
        u, st = solver.solve(b, tol=tol, allow_noconv=True)
        ctx.stats = st
        ctx.solver = solver
        ctx.tol = tol
        ctx.eps_device = eps.device
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        s = ctx.solver
        lam, _ = s.solve(torch.conj(grad_u).resolve_conj().contiguous(), tol=ctx.tol, allow_noconv=True)
        g = s.grad_eps(u, lam)
        return g.to(device=ctx.eps_device, dtype=torch.float64), None, None, None, None


def solver_k(solver) -> float:
    return solver.k


def make_solver(device: int, base_n: int, leaves, p, k: float, eps):
    from .ddh import DDH
    s = DDH(device)
    s.set_mesh(base_n, leaves, p)
    s.k = float(k)
    s.set_coefficients(k, eps)
    return s


class PointEval(torch.autograd.Function):
    """y = E u: field values at fixed points (E real, so the backward is the injection E^T)."""

    @staticmethod
    def forward(ctx, u: torch.Tensor, solver, xy):
        ctx.solver = solver
        ctx.xy = xy
        return solver.eval_points(xy, u)

    @staticmethod
    def backward(ctx, grad_y):
        return ctx.solver.inject_points(ctx.xy, grad_y.contiguous()), None, None
