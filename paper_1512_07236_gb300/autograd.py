"""torch.autograd.Function over the fixed-iteration GCP recursion.

GCPFunction.apply(H, N, fixed_iters, ckpt_every) -> (D, E) runs exactly
`fixed_iters` FP64 steps of the recursion from the canonical guess
(gcp_solve) and, on backward, calls gcp_backward, the hand-written adjoint
(checkpointed reverse mode through every step and through the guess).
Argument marshalling only; the arithmetic is in libgcp.
"""
from __future__ import annotations

import torch

from . import gcp

__all__ = ["GCPFunction", "gcp_density"]


class GCPFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, N, fixed_iters=40, ckpt_every=8):
        if H.dtype != torch.float64:
            raise TypeError("GCPFunction runs the FP64 recursion: pass a float64 H")
        H = H.contiguous()
        D, info = gcp.default_solver().solve(H, int(N), prec="fp64",
                                             fixed_iters=int(fixed_iters))
        E = torch.tensor(info["energy"], dtype=H.dtype, device=H.device)
        ctx.save_for_backward(H)
        ctx.N, ctx.K, ctx.ck = int(N), int(fixed_iters), int(ckpt_every)
        return D, E

    @staticmethod
    def backward(ctx, gD, gE):
        (H,) = ctx.saved_tensors
        G = None
        if gD is not None:
            G = (0.5 * (gD + gD.transpose(0, 1))).contiguous()  # D is symmetric
        g_E = float(gE) if gE is not None else 0.0
        dH = gcp.default_solver().backward(H, ctx.N, ctx.K, G_D=G, g_E=g_E,
                                           ckpt_every=ctx.ck)
        return dH, None, None, None


def gcp_density(H, N, fixed_iters=40, ckpt_every=8):
    """Differentiable (D, E) after `fixed_iters` steps from the guess of H."""
    return GCPFunction.apply(H, N, fixed_iters, ckpt_every)
