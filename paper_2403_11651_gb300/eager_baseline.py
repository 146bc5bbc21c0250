"""One overfitting iteration written with plain PyTorch eager operations: the comparison
baseline that bench.py times beside the CUDA library on the same GPU.  No path of the
library calls it; it exists to show what the hand-written kernels gain over stock
framework operations.

The iteration is the same as the library's (Sec. II, eq. (1); Table 1): quantisation by
additive noise (or rint with a straight-through gradient), the ARM over every latent of
the 7 levels (the N nearest causal neighbours, 0 outside a level), the Laplace rate with
the scale clamped to [1e-2, 1e3] and the bin probability floored at 2^-16, every level
brought to full resolution by stride-2 transposed convolutions reading their input
clamp-to-edge, the 1x1 synthesis layers and the residual 3x3 layers with replicated
borders, D + lambda R, autograd's backward and torch.optim.Adam (beta 0.9 / 0.999,
eps 1e-8).  It is written for the GPU: all levels' contexts go through one MLP call,
and each upsampling step is one conv_transpose2d.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as F

LEVELS = 7


def causal_offsets(n: int):
    """The n causal neighbours (dy < 0, or dy = 0 and dx < 0) nearest in Euclidean
    distance, ties broken by smaller |dy| then smaller dx; returned in raster order."""
    cands = [(dy, dx) for dy in range(-6, 1) for dx in range(-6, 7) if dy < 0 or dx < 0]
    cands.sort(key=lambda o: (o[0] ** 2 + o[1] ** 2, abs(o[0]), o[1]))
    return sorted(cands[:n])


def level_shapes(H: int, W: int):
    return [((H + (1 << l) - 1) >> l, (W + (1 << l) - 1) >> l) for l in range(LEVELS)]


class EagerIteration:
    """State (latents, parameters, Adam) of one image on `device`; step() is one iteration.

    cfg: a configuration dict (the keys of configs/*.json); init: named initial parameters
    (the names of synthetic.initial_parameters); rgb: H x W x 3 uint8."""

    def __init__(self, rgb: np.ndarray, cfg: dict, init: dict, device, dtype=torch.float32):
        self.cfg, self.dev, self.dt = cfg, torch.device(device), dtype
        H, W = rgb.shape[:2]
        self.H, self.W = H, W
        self.shapes = level_shapes(H, W)
        self.x = torch.tensor(np.transpose(rgb, (2, 0, 1)) / 255.0, dtype=dtype, device=self.dev)
        self.y = [torch.zeros(h, w, dtype=dtype, device=self.dev, requires_grad=True)
                  for h, w in self.shapes]
        self.P = {k: torch.tensor(np.asarray(v, np.float64), dtype=dtype, device=self.dev,
                                  requires_grad=True) for k, v in init.items()}
        self.offsets = causal_offsets(cfg["arm_ctx"])
        self.reach = max(max(-dy, abs(dx)) for dy, dx in self.offsets)
        self.opt = torch.optim.Adam(self.y + list(self.P.values()), lr=cfg["lr"],
                                    betas=(0.9, 0.999), eps=1e-8)
        self.t = 0
        self.ste_start = int(round(cfg["total_iters"] * (1.0 - cfg["ste_frac"])))

    # ---------------------------------------------------------------- forward pieces
    def _contexts(self, yhat):
        """[n_latents, N]: every latent's causal context, level after level."""
        r, out = self.reach, []
        for yl in yhat:
            h, w = yl.shape
            p = F.pad(yl, (r, r, r, 0))
            out.append(torch.stack([p[r + dy:r + dy + h, r + dx:r + dx + w].reshape(-1)
                                    for dy, dx in self.offsets], 1))
        return torch.cat(out, 0)

    def _bits(self, yhat):
        P, nl = self.P, self.cfg["arm_layers"]
        h = self._contexts(yhat)
        for i in range(nl):
            h = h + torch.relu(F.linear(h, P[f"arm.w{i}"], P[f"arm.b{i}"]))
        mu_s = F.linear(h, P["arm.wout"], P["arm.bout"])
        v = torch.cat([yl.reshape(-1) for yl in yhat])
        b = torch.exp(torch.clamp(mu_s[:, 1], math.log(1e-2), math.log(1e3)))
        d = v - mu_s[:, 0]
        # mass of [v - 1/2, v + 1/2]: both ends on one side of mu, or mu inside the bin
        one_side = 0.5 * torch.exp(-(torch.clamp(d.abs(), min=0.5) - 0.5) / b) \
            * -torch.expm1(-1.0 / b)
        dc = torch.clamp(d, -0.5, 0.5)
        straddle = -0.5 * (torch.expm1(-(0.5 + dc) / b) + torch.expm1(-(0.5 - dc) / b))
        p = torch.where(d.abs() >= 0.5, one_side, straddle)
        return -torch.log2(torch.clamp(p, min=2.0 ** -16)).sum()

    def _up2(self, a, f, out_h, out_w):
        """Stride-2 transposed convolution of a (clamp-to-edge inputs), output phase
        centred (a k x k filter, offset k/2 - 1), cropped to out_h x out_w."""
        k = f.shape[-1]
        p = k // 4
        ap = F.pad(a[None, None], (p, p, p, p), mode="replicate")
        full = F.conv_transpose2d(ap, f[None, None], stride=2)[0, 0]
        o = k // 2 - 1 + 2 * p
        return full[o:o + out_h, o:o + out_w]

    def _synthesis_input(self, yhat):
        per_level = self.cfg["up_per_level"]
        feats = [yhat[0]]
        for l in range(1, LEVELS):
            f = self.P[f"up.f{l}"] if per_level else self.P["up.f"]
            a = yhat[l]
            for j in range(l - 1, -1, -1):
                a = self._up2(a, f, *self.shapes[j])
            feats.append(a)
        return torch.stack(feats)

    def _synthesis(self, feat):
        P, n3 = self.P, self.cfg["syn_res3x3"]
        h = torch.relu(F.conv2d(feat[None], P["syn.wa"][:, :, None, None], P["syn.ba"]))
        h = torch.relu(F.conv2d(h, P["syn.wb"][:, :, None, None], P["syn.bb"]))
        for i in range(n3):
            z = F.conv2d(F.pad(h, (1, 1, 1, 1), mode="replicate"), P[f"syn.w3_{i}"],
                         P[f"syn.b3_{i}"])
            h = h + (torch.relu(z) if i < n3 - 1 else z)
        return h[0]

    def loss(self, noise=None, hard=None):
        """(loss, D, R_bpp) at the current state; noise: per-level tensors in
        [-1/2, 1/2) (drawn on the device when None); hard: rint + straight-through."""
        if hard is None:
            hard = self.t >= self.ste_start
        if hard:
            yhat = [yl + (torch.round(yl) - yl).detach() for yl in self.y]
        else:
            if noise is None:
                noise = [torch.rand_like(yl) - 0.5 for yl in self.y]
            yhat = [yl + u for yl, u in zip(self.y, noise)]
        R = self._bits(yhat) / (self.H * self.W)
        D = torch.mean((self._synthesis(self._synthesis_input(yhat)) - self.x) ** 2)
        return D + self.cfg["lam"] * R, D, R

    def step(self, noise=None):
        """One iteration: forward, backward, Adam."""
        self.opt.zero_grad(set_to_none=True)
        L, D, R = self.loss(noise)
        L.backward()
        self.opt.step()
        self.t += 1
        return L, D, R
