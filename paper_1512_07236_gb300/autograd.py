"""torch.autograd.Function over the fixed-iteration GCP recursion.

GCPFunction.apply(H, N, fixed_iters, ckpt_every) -> (D, E) runs exactly
`fixed_iters` steps of the recursion from the canonical guess (gcp_solve)
and, on backward, calls gcp_backward, the hand-written adjoint (checkpointed
reverse mode through every step and through the guess).  A float64 H runs
the FP64 recursion and adjoint; a float32 H the GCP_FP32 ones (split-FP16
tensor-core products, FP32 state), D and the gradient in float32.
Argument marshalling only; the arithmetic is in libgcp.
"""
from __future__ import annotations

import torch

from . import gcp

__all__ = ["GCPFunction", "gcp_density"]


class GCPFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, N, fixed_iters=40, ckpt_every=8):
        if H.dtype not in (torch.float64, torch.float32):
            raise TypeError("GCPFunction takes a float64 (FP64 recursion) or float32 "
                            "(FP32 tensor-core recursion) H")
        H = H.contiguous()
        prec = "fp64" if H.dtype == torch.float64 else "fp32"
        D, info = gcp.default_solver().solve(H, int(N), prec=prec, out_dtype=H.dtype,
                                             fixed_iters=int(fixed_iters))
        E = torch.tensor(info["energy"], dtype=H.dtype, device=H.device)
        ctx.save_for_backward(H)
        ctx.N, ctx.K, ctx.ck, ctx.prec = int(N), int(fixed_iters), int(ckpt_every), prec
        return D, E

    @staticmethod
    def backward(ctx, gD, gE):
        (H,) = ctx.saved_tensors
        G = None
        if gD is not None:
            G = (0.5 * (gD + gD.transpose(0, 1))).contiguous()  # D is symmetric
        g_E = float(gE) if gE is not None else 0.0
        dH = gcp.default_solver().backward(H, ctx.N, ctx.K, G_D=G, g_E=g_E,
                                           ckpt_every=ctx.ck, prec=ctx.prec)
        return dH, None, None, None


def gcp_density(H, N, fixed_iters=40, ckpt_every=8):
    """Differentiable (D, E) after `fixed_iters` steps from the guess of H."""
    return GCPFunction.apply(H, N, fixed_iters, ckpt_every)
