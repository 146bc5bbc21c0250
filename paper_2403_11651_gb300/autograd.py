"""``torch.autograd.Function`` over the library's hand-written backward (argument
marshalling only: the forward and the backward of the pass both run in the CUDA library).

``CoolChicIter.apply(handle, y, params, noise, hard)`` returns the loss of eq. (1),
D + lambda R (computed by the library with the context's lambda), of one pass of the context ``handle`` over the latents ``y`` (flat latent
order) and the decoder parameters ``params`` (flat parameter order); its backward returns
dL/dy and dL/dparams, which the library's backward (the adjoints of the synthesis, the
upsampling and the ARM, with the straight-through or noise quantisation rule of the
pass) computed in the same call.  ``noise``: explicit quantisation noise (flat latent
order) or None for the context's own noise of its current iteration; ``hard``: 1 rint
latents with straight-through gradients, 0 noise, -1 the context's schedule.

The context should be created on the stream the tensors are produced on (for example
``torch.cuda.current_stream()`` passed to ``cc_init_image``); the call synchronises it.
"""
from __future__ import annotations

import torch

from . import coolchic as cc


class CoolChicIter(torch.autograd.Function):
    @staticmethod
    def forward(fctx, handle, y: torch.Tensor, params: torch.Tensor, noise=None,
                hard: int = -1):
        if not (y.is_cuda and params.is_cuda):
            raise ValueError("CoolChicIter: y and params must be CUDA tensors")
        y32 = y.detach().to(torch.float32).contiguous()
        p32 = params.detach().to(torch.float32).contiguous()
        cc.cc_set_latents(handle, y32)
        cc.cc_set_params(handle, p32)
        grads = torch.empty(y32.numel() + p32.numel(), dtype=torch.float32, device=y.device)
        _, _, _, loss = cc.cc_forward_backward(handle, grads.numel(), noise, int(hard), grads,
                                               with_loss=True)
        fctx.save_for_backward(grads)
        fctx.n_lat = y32.numel()
        fctx.dtypes = (y.dtype, params.dtype)
        return torch.tensor(loss, dtype=torch.float64, device=y.device)

    @staticmethod
    def backward(fctx, grad_loss):
        (grads,) = fctx.saved_tensors
        s = grad_loss.to(torch.float32)
        gy = (s * grads[:fctx.n_lat]).to(fctx.dtypes[0])
        gp = (s * grads[fctx.n_lat:]).to(fctx.dtypes[1])
        return None, gy, gp, None, None


def coolchic_loss(handle, y: torch.Tensor, params: torch.Tensor, noise=None,
                  hard: int = -1) -> torch.Tensor:
    """D + lambda R of one pass, differentiable in y and params (CoolChicIter)."""
    return CoolChicIter.apply(handle, y, params, noise, hard)
