"""torch.autograd wrapper: u = solve(mu^{-1}, omega) with a backward pass
through the library's adjoint (thm_adjoint).

PyTorch hands backward the gradient 2 dL/d(conj u) of a real loss; the
adjoint takes a = dL/du = conj(grad_u) / 2.  The backward pass reuses the
assembled operators and the stored solution u (no Krylov bases are kept).
"""
from __future__ import annotations

import torch

from ._binding import System


class ThmSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu_inv, omega, mesh, kappa, pol, direction, opts):
        om = float(omega)
        sysg = System(mesh, mu_inv.detach(), om, kappa, pol, direction)
        u, st = sysg.solve(**opts)
        ctx.sysg = sysg
        ctx.opts = opts
        ctx.omega_is_tensor = isinstance(omega, torch.Tensor)
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        a = (grad_u.conj() * 0.5).contiguous()
        g_mu, g_w, _ = ctx.sysg.adjoint(u, a, **ctx.opts)
        gw = torch.tensor(g_w, dtype=torch.float64, device=u.device) if ctx.omega_is_tensor else None
        return g_mu, gw, None, None, None, None, None


def solve(mesh, mu_inv, omega, kappa, pol, direction, mode="fp64", rtol=1e-10, **kw):
    """Differentiable solve: mu_inv a float64 CUDA tensor [n_cell] (may require
    grad), omega a float or a 0-d tensor (may require grad)."""
    opts = dict(mode=mode, rtol=rtol, **kw)
    return ThmSolve.apply(mu_inv, omega, mesh, kappa, pol, direction, opts)
