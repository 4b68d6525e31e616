"""torch.autograd.Function around the GPU Stokes solve.

forward:  (f, nu) -> x = [u; p] solving K(nu) x = [f; 0] (pressure zero-mean)
backward: K is symmetric (Sec. 5), so the adjoint is one more preconditioned
          MINRES solve K lambda = [dL/du; P^T dL/dp] (gb_solve_adjoint), and
          dL/df = lambda_u,  dL/dnu = -sum_k lambda_u^T A_0 u  (A_h = nu A_0).
"""
from __future__ import annotations

import torch


class StokesSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, nu, solver, opts):
        """f: (k, n_u) or (n_u,) float64 CUDA load vectors; nu: 0-d float64
        tensor; solver: an assembled and factored gbstokes.Stokes; opts: dict
        of solve options.  Re-assembles and re-factors if nu changed."""
        nuv = float(nu)
        if solver.nu is None or solver.nu != nuv:
            solver.assemble(nuv)
            solver.factor_ic0()
        single = f.dim() == 1
        f2 = f.reshape(-1, solver.n_u)
        rhs = torch.zeros(f2.shape[0], solver.n, dtype=torch.float64, device=f.device)
        rhs[:, :solver.n_u] = f2
        x, _ = solver.solve(rhs, **opts)
        ctx.solver, ctx.opts, ctx.single = solver, opts, single
        ctx.save_for_backward(x)
        return x[0] if single else x

    @staticmethod
    def backward(ctx, grad_x):
        (x,) = ctx.saved_tensors
        solver = ctx.solver
        g = grad_x.reshape(-1, solver.n).contiguous().to(torch.float64)
        lam, _ = solver.solve_adjoint(g, **ctx.opts)
        grad_f = lam[:, :solver.n_u].clone()
        dnu = solver.dnu(lam, x)
        grad_nu = torch.tensor(float(dnu.sum()), dtype=torch.float64, device=x.device)
        if ctx.single:
            grad_f = grad_f[0]
        return grad_f, grad_nu, None, None


def stokes_solve(f, nu, solver, **opts):
    return StokesSolve.apply(f, nu, solver, opts)
