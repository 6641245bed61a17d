"""torch.autograd.Function for the plane-wave Helmholtz solve as a function of the element
permittivities and the wavenumber.  Forward: set eps and k, factor, solve (all in libddh).
Backward: the transposed adjoint system A^T lam = conj(G) is an ordinary solve on the same
kernels (A is complex symmetric), then the per-element gradient-accumulation kernel gives
dJ/deps_e = k^2 (h_e/2)^2 Re(lam_e^T M_e u_e), and ddh_grad_k gives dJ/dk through the mass
term, the Robin term and the plane-wave load.  A forward or adjoint solve that misses its
tolerance raises (ddh.DDHError with ERR_NO_CONVERGENCE) unless allow_noconv is set.
"""
from __future__ import annotations

import torch


def _as_float(k) -> float:
    return float(k.detach().cpu().item()) if isinstance(k, torch.Tensor) else float(k)


class PlaneWaveSolve(torch.autograd.Function):
    """u = A(eps, k)^-1 b(k) for the plane waves of angles `thetas`.

    apply(eps, k, solver, thetas, tol=1e-12, factor_opts=None, allow_noconv=False):
    eps is a float64 tensor [n_elem]; k a float64 scalar tensor (or a float, then no dJ/dk)."""

    @staticmethod
    def forward(ctx, eps: torch.Tensor, k, solver, thetas, tol: float = 1e-12, factor_opts: dict | None = None,
                allow_noconv: bool = False):
        kv = _as_float(k)
        solver.k = kv
        solver.set_coefficients(kv, eps.detach().cpu().double().numpy())
        solver.factor(**(factor_opts or {}))
        b = solver.rhs_planewave(thetas)
        u, st = solver.solve(b, tol=tol, allow_noconv=allow_noconv)
        ctx.stats = st
        ctx.solver = solver
        ctx.tol = tol
        ctx.thetas = thetas
        ctx.allow_noconv = allow_noconv
        ctx.eps_device = eps.device
        ctx.k_tensor = isinstance(k, torch.Tensor)
        ctx.k_device = k.device if ctx.k_tensor else None
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        s = ctx.solver
        lam, _ = s.solve(torch.conj(grad_u).resolve_conj().contiguous(), tol=ctx.tol, allow_noconv=ctx.allow_noconv)
        g_eps = g_k = None
        if ctx.needs_input_grad[0]:
            g_eps = s.grad_eps(u, lam).to(device=ctx.eps_device, dtype=torch.float64)
        if ctx.k_tensor and ctx.needs_input_grad[1]:
            g_k = torch.tensor(s.grad_k(u, lam, ctx.thetas), dtype=torch.float64, device=ctx.k_device)
        return g_eps, g_k, None, None, None, None, None


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
