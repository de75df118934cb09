"""torch.autograd.Function over libcld: Gamma = logdet estimate of the CSR
matrix with the given values, differentiable with respect to the values.

The forward calls cld_grad when a gradient is needed (it returns Gamma and
dGamma/dval together) and cld_estimate otherwise; the backward scales the
stored gradient by the incoming scalar.  The spectral interval and the probes
are held fixed, so the gradient is that of the estimator as a function of the
stored values."""
from __future__ import annotations

import torch

from .api import CsrLogdet


class CldLogdet(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, rowptr, col, n, M, seed, interval, checkpoint):
        dtype = {torch.float32: "f32", torch.float64: "f64", torch.bfloat16: "bf16"}[values.dtype]
        m = CsrLogdet(rowptr, col, values.detach(), dtype=dtype, device=values.device)
        try:
            m.set_interval(*interval)
            m.set_grad_checkpoint(checkpoint)
            if ctx.needs_input_grad[0]:
                g, G = m.grad(n, M, seed)
                ctx.save_for_backward(G)
            else:
                g = m.estimate(n, M, seed)["logdet"]
        finally:
            m.close()
        return torch.tensor(g, dtype=torch.float64, device=values.device)

    @staticmethod
    def backward(ctx, grad_out):
        (G,) = ctx.saved_tensors
        return (grad_out * G.double()).to(G.dtype), None, None, None, None, None, None, None


def logdet(values, rowptr, col, n: int, M: int, seed: int = 0, interval=(None, None), checkpoint: int = 0):
    """Differentiable estimate; ``interval`` = (a, b) enclosing the spectrum;
    ``checkpoint`` = 0 keeps every w_j for the backward, K >= 2 keeps pairs
    every K steps and recomputes (see cld_set_grad_checkpoint)."""
    return CldLogdet.apply(values, rowptr, col, n, M, seed, tuple(interval), int(checkpoint))
