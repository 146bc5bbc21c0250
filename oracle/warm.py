"""Warm-start predictor (image -> latent pyramid) in FP64 -- TEST INFRASTRUCTURE ONLY.

Same import rule as ``oracle.coolchic``: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module; the product path runs the CUDA library.

The paper's encoder starts every image from zero latents and spends its iterations
finding them; Sec. IV-B (the non-overfitted variant) predicts the latents with an analysis
network trained on a dataset, and Sec. V proposes, as future work, fine-tuning such a
prediction per image instead of overfitting from scratch.  This predictor is the small version of that idea: a stack of four 3x3 stride-2
convolutions with 32 channels and ReLU (zero padding 1) whose outputs at 1/2 .. 1/16 of
the image resolution give latent levels 1 .. 4 through 1x1 convolutions, plus one 3x3
convolution of the image (stride 1) for level 0; levels 5 and 6 start at 0.  Trained by
the mean squared error against latents this project's encoder reached, summed over the
predicted levels (each level's mean).  Written with torch's conv2d as the convolution
step (its definition: out[co, y, x] = b[co] + sum over ci, ky, kx of
w[co, ci, ky, kx] in[ci, s y + ky - 1, s x + kx - 1]).
"""
from __future__ import annotations

import torch
import torch.nn.functional as F

DT = torch.float64
CH = 32
LEVELS_PREDICTED = 5     # levels 0 .. 4


def param_shapes():
    """Ordered (name, shape) list (flat parameter order of the CUDA predictor)."""
    out = [("c1.w", (CH, 3, 3, 3)), ("c1.b", (CH,))]
    for i in (2, 3, 4):
        out += [(f"c{i}.w", (CH, CH, 3, 3)), (f"c{i}.b", (CH,))]
    for i in (1, 2, 3, 4):
        out += [(f"h{i}.w", (1, CH, 1, 1)), (f"h{i}.b", (1,))]
    out += [("h0.w", (1, 3, 3, 3)), ("h0.b", (1,))]
    return out


def to_bf16(t: torch.Tensor) -> torch.Tensor:
    """t rounded to the nearest BF16 value (8 significand bits, ties to even), kept in FP64."""
    return t.to(torch.bfloat16).to(DT)


class ConvBF16(torch.autograd.Function):
    """conv2d with stride 2 and zero padding 1 whose operands are rounded to BF16 wherever
    the convolution is evaluated: the forward pass rounds the input and the weights, the
    backward pass rounds the output gradient and uses the rounded input and weights for the
    input gradient, the weight gradient and the bias gradient (the sum of the rounded output
    gradient).  Every sum is FP64.  This is the arithmetic of the tensor-core layers
    (BF16 operands, wide accumulation)."""

    @staticmethod
    def forward(ctx, a, w, b):
        ab, wb = to_bf16(a), to_bf16(w)
        ctx.save_for_backward(ab, wb)
        return F.conv2d(ab, wb, b, stride=2, padding=1)

    @staticmethod
    def backward(ctx, g):
        ab, wb = ctx.saved_tensors
        gb = to_bf16(g)
        da = torch.nn.grad.conv2d_input(ab.shape, wb, gb, stride=2, padding=1)
        dw = torch.nn.grad.conv2d_weight(ab, wb.shape, gb, stride=2, padding=1)
        return da, dw, gb.sum(dim=(0, 2, 3))


def forward(x: torch.Tensor, P: dict, bf16: bool = False):
    """x: [3, H, W] -> [latent level 0 .. 4] (each [h_l, w_l]).  With bf16, the 32-to-32
    channel convolutions (conv 2 .. 4) take BF16-rounded operands (ConvBF16)."""
    a = x.unsqueeze(0)
    lv = [F.conv2d(a, P["h0.w"], P["h0.b"], stride=1, padding=1)[0, 0]]
    for i in (1, 2, 3, 4):
        if bf16 and i > 1:
            z = ConvBF16.apply(a, P[f"c{i}.w"], P[f"c{i}.b"])
        else:
            z = F.conv2d(a, P[f"c{i}.w"], P[f"c{i}.b"], stride=2, padding=1)
        a = torch.relu(z)
        lv.append(F.conv2d(a, P[f"h{i}.w"], P[f"h{i}.b"])[0, 0])
    return lv


def loss(x: torch.Tensor, P: dict, targets, bf16: bool = False):
    """sum over the predicted levels of the mean squared error."""
    return sum(((p - t) ** 2).mean() for p, t in zip(forward(x, P, bf16), targets))
