"""torch.autograd.Function over the library's log-likelihood and its hand-written adjoint.

forward  : exa_loglik (no gradient needed) or exa_loglik_grad (a gradient of theta is
           needed), which returns l and dl/dtheta from one factorisation (the adjoint
           1/2 a^T dSigma a - 1/2 tr(Sigma^-1 dSigma), a = Sigma^-1 z), both in the
           caller's precision `prec`; a precision the library's gradient does not offer
           raises instead of being replaced by another.
backward : grad_output * dl/dtheta.
Only the three covariance parameters are differentiable; locations and data are
treated as constants.
"""
from __future__ import annotations

import torch

from . import Context


class MaternLogLik(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, locs, z, exa_ctx, prec):
        th = [float(v) for v in theta.detach().cpu().tolist()]
        if fctx.needs_input_grad[0]:
            l, g = exa_ctx.loglik_grad(locs, z, th, prec)
            fctx.save_for_backward(torch.tensor(g, dtype=theta.dtype, device=theta.device))
        else:
            l = exa_ctx.loglik(locs, z, th, prec)
        return torch.tensor(l, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(fctx, grad_out):
        (g,) = fctx.saved_tensors
        return grad_out * g, None, None, None, None


def loglik(theta: torch.Tensor, locs: torch.Tensor, z: torch.Tensor, ctx: Context | None = None,
           prec: int | None = None) -> torch.Tensor:
    """l(theta) as a differentiable scalar tensor (theta: 3 float64 values).  prec=None: the context's
    default (EXA_PREC from the environment, else EXA_FP64)."""
    own = ctx is None
    c = Context() if own else ctx
    try:
        return MaternLogLik.apply(theta, locs, z, c, prec)
    finally:
        if own:
            c.close()
