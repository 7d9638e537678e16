"""PyTorch autograd wrapper of the modelling operator.

``propagate(ctx, v, wavelet)`` returns the seismograms d = R A(v)^{-1} f (Eq. "fwi",
"wave"); its backward is the library's exact discrete adjoint-state gradient
(Eq. "FWI_lambda", "gradient"): a vector-Jacobian product g = (dd/dv)^T (dL/dd) computed
by esi_gradient with the upstream gradient as the adjoint source and checkpointed
recomputation of the forward states (every ``ckpt_every`` steps, stored in FP32, FP16 or
BF16 with a per-snapshot scale).  Both directions run in libesi's kernels; this module
only routes tensors.

The sponge profile is fixed when the context is created (its reference velocity does not
follow v), so the gradient is exact for the discrete operator as a function of v.
"""
from __future__ import annotations

import torch


class ESIPropagate(torch.autograd.Function):
    @staticmethod
    def forward(fctx, v, wavelet, ctx, ckpt_every: int = 20, ckpt: str = "bf16"):
        ctx.set_velocity(v.detach().contiguous())
        d = ctx.forward(wavelet=wavelet.detach().contiguous())
        fctx.esi = ctx
        fctx.opts = (int(ckpt_every), ckpt)
        fctx.save_for_backward(v, wavelet)
        return d

    @staticmethod
    def backward(fctx, grad_d):
        v, wavelet = fctx.saved_tensors
        ctx = fctx.esi
        ckpt_every, ckpt = fctx.opts
        ctx.set_velocity(v.detach().contiguous())
        g, _ = ctx.gradient(wavelet=wavelet.detach().contiguous(),
                            adj_src=grad_d.detach().contiguous(), param="v",
                            ckpt_every=ckpt_every, ckpt=ckpt)
        return g, None, None, None, None


def propagate(ctx, v, wavelet, ckpt_every: int = 20, ckpt: str = "bf16"):
    """Differentiable forward modelling: traces as a function of the velocity v."""
    return ESIPropagate.apply(v, wavelet, ctx, ckpt_every, ckpt)
