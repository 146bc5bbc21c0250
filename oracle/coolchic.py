"""FP64 CPU oracle of one Cool-chic overfitting iteration -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package's ``__graft_entry__.smoke()`` check and the CPU-baseline leg of
``bench.py`` may import this module.  The product path never does: it runs the CUDA library.

It restates, in float64 and plain PyTorch CPU ops, what one iteration of the method computes
(Sec. II of Blard et al., "Overfitted image coding at reduced complexity", eq. (1)):

    loss = D(x, f_theta(f_upsilon(y_hat))) + lambda * R(y_hat),   R = -log2 p_psi(y_hat)

over the L = 7 latent grids y_hat_l of size H/2^l x W/2^l (Sec. II "Decoding", item i),
with the auto-regressive model p_psi (item ii), the linear learned upsampling f_upsilon and
the synthesis f_theta (item iii) whose layer list is Table 1; then its gradient (computed by
autograd, the derivative's definition) and one Adam step (Kingma & Ba, used in Sec. IV-B).

Readings taken where the paper defers to earlier Cool-chic / C3 work (each one is also
listed with its reason in the design notes of the repository):

* ARM context: the N causal neighbours (dy < 0, or dy = 0 and dx < 0) nearest in
  Euclidean distance, ties broken by smaller |dy| then smaller dx, kept in raster order;
  positions outside the grid read 0; each level is modelled on its own.
* Residual layers ("LinR", "ConvR" in Table 1): out = in + act(W in + b), act = ReLU
  except for the last layer of a module, which has none (Table 1 caption).  The 1x1 C->3
  synthesis layer is not the last one, so it has a ReLU.
* Laplace model: the ARM's two outputs are (mu, s), scale b = exp(clamp(s, ln 1e-2,
  ln 1e3)); P(y_hat) = F(y_hat + 1/2) - F(y_hat - 1/2) evaluated in a cancellation-free
  form; rate per latent -log2(max(P, 2^-16)).
* Upsampling of level l >= 1: l repeated stride-2 k x k transposed convolutions with the
  level's filter (one filter per level, or one shared filter for the Table 1 parameter
  count); inputs read with clamp-to-edge, phases centred as in align_corners=False
  resampling, outputs cropped to the next level's size.
* 3x3 convolutions read with replicate padding.
* D = mean of the 3HW squared errors; R = total bits / (H W) (bits per pixel).
* Quantisation proxy: y_hat = y + u with uniform noise u, or y_hat = rint(y) with a
  straight-through gradient in the last part of training.  With a soft-rounding
  temperature T > 0 (C3's proxy, to which Sec. II "Encoding" refers), the noise phase uses
  y_hat = s_T(s_T(y) + u) with the soft rounding
  s_T(x) = floor(x) + 1/2 + tanh((x - floor(x) - 1/2) / T) / (2 tanh(1 / (2T))),
  differentiated through both soft roundings.
* Adam: beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, one learning rate for all.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch
import torch.nn.functional as F

from . import philox

DT = torch.float64
LOG_B_MIN = math.log(1e-2)
LOG_B_MAX = math.log(1e3)
P_MIN = 2.0 ** -16
ADAM_BETA1, ADAM_BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


@dataclass(frozen=True)
class Arch:
    """Decoder architecture in Table 1 notation."""
    levels: int = 7
    arm_ctx: int = 24        # N: context size = ARM hidden width (LinR layers are N -> N)
    arm_layers: int = 2      # number of N-N-LinR layers before the N-2-Lin output layer
    up_kernel: int = 8       # k of the 1-1-TConv-k layer
    up_per_level: bool = True
    syn_hidden: int = 40     # C of the 7-C-Conv-1 layer
    syn_res3x3: int = 2      # number of 3-3-ConvR-3 layers


@dataclass(frozen=True)
class Train:
    lam: float = 1e-3
    lr: float = 1e-2
    total_iters: int = 10000
    ste_frac: float = 0.0    # last fraction of iterations with straight-through rounding
    seed: int = 0
    soft_temp: float = 0.0   # C3 soft-rounding temperature of the noise phase; 0: y + u

    @property
    def ste_start(self) -> int:
        return int(round(self.total_iters * (1.0 - self.ste_frac)))


# --------------------------------------------------------------------------------------
# Geometry (Sec. II "Decoding", item i)
# --------------------------------------------------------------------------------------

def level_shapes(H: int, W: int, levels: int = 7):
    """Level l grid is ceil(H / 2^l) x ceil(W / 2^l)."""
    return [(-(-H // (1 << l)), -(-W // (1 << l))) for l in range(levels)]


def causal_offsets(n: int):
    """The n nearest causal neighbours (dy, dx), in raster order."""
    reach = 6
    cands = [(dy, dx) for dy in range(-reach, 1) for dx in range(-reach, reach + 1)
             if dy < 0 or dx < 0]
    cands.sort(key=lambda o: (o[0] * o[0] + o[1] * o[1], abs(o[0]), o[1]))
    return sorted(cands[:n])


# --------------------------------------------------------------------------------------
# Parameters (Table 1)
# --------------------------------------------------------------------------------------

def param_shapes(arch: Arch):
    """Ordered (name, shape) list.  Linear weights are (out, in); 3x3 weights (out, in, 3, 3)."""
    n = arch.arm_ctx
    out = []
    for i in range(arch.arm_layers):
        out += [(f"arm.w{i}", (n, n)), (f"arm.b{i}", (n,))]
    out += [("arm.wout", (2, n)), ("arm.bout", (2,))]
    k = arch.up_kernel
    if arch.up_per_level:
        out += [(f"up.f{l}", (k, k)) for l in range(1, arch.levels)]
    else:
        out += [("up.f", (k, k))]
    c = arch.syn_hidden
    out += [("syn.wa", (c, arch.levels)), ("syn.ba", (c,)),
            ("syn.wb", (3, c)), ("syn.bb", (3,))]
    for i in range(arch.syn_res3x3):
        out += [(f"syn.w3_{i}", (3, 3, 3, 3)), (f"syn.b3_{i}", (3,))]
    return out


def param_count(arch: Arch) -> int:
    return sum(int(np.prod(s)) for _, s in param_shapes(arch))


def macs_per_pixel(arch: Arch, H: int | None = None, W: int | None = None) -> dict:
    """Decoder multiplications per pixel, split by module (Fig. 4a's breakdown).

    With H, W given the counts are exact for that image; otherwise the asymptotic ratios
    (sum over l of 4^-l latents per pixel) are used.
    """
    n, k, c = arch.arm_ctx, arch.up_kernel, arch.syn_hidden
    arm_per_latent = arch.arm_layers * n * n + 2 * n
    taps = (k // 2) ** 2
    if H is None:
        lat = sum(4.0 ** -l for l in range(arch.levels))
        ups = sum(sum(4.0 ** -j for j in range(l)) for l in range(1, arch.levels))
    else:
        sh = level_shapes(H, W, arch.levels)
        hw = float(H * W)
        lat = sum(h * w for h, w in sh) / hw
        ups = sum(sum(sh[j][0] * sh[j][1] for j in range(l))
                  for l in range(1, arch.levels)) / hw
    syn = arch.levels * c + 3 * c + arch.syn_res3x3 * 81
    res = {"arm": arm_per_latent * lat, "upsampling": taps * ups, "synthesis": float(syn)}
    res["total"] = res["arm"] + res["upsampling"] + res["synthesis"]
    return res


def params_from_numpy(named: dict, arch: Arch, requires_grad=True) -> dict:
    P = {}
    for name, shape in param_shapes(arch):
        a = np.asarray(named[name], dtype=np.float64)
        assert a.shape == tuple(shape), (name, a.shape, shape)
        P[name] = torch.tensor(a, dtype=DT, requires_grad=requires_grad)
    return P


# --------------------------------------------------------------------------------------
# Quantisation proxy (Sec. II "Encoding")
# --------------------------------------------------------------------------------------

def soft_round(x: torch.Tensor, T: float) -> torch.Tensor:
    """C3's soft rounding with temperature T: integers and half-integers are fixed points,
    it tends to rounding as T -> 0 and to the identity as T grows."""
    f = torch.floor(x)
    return f + 0.5 + 0.5 * torch.tanh((x - f - 0.5) / T) / math.tanh(0.5 / T)


def quantize(y: torch.Tensor, u, hard: bool, soft_temp: float = 0.0) -> torch.Tensor:
    """Noise: y + u, or s_T(s_T(y) + u) with a soft-rounding temperature T = soft_temp > 0.
    Hard: rint(y) (round half to even) with the identity as gradient."""
    if hard:
        return y + (torch.round(y) - y).detach()
    if soft_temp > 0.0:
        return soft_round(soft_round(y, soft_temp) + u, soft_temp)
    return y + u


# --------------------------------------------------------------------------------------
# ARM p_psi (Sec. II "Decoding" item ii; Table 1 "ARM")
# --------------------------------------------------------------------------------------

def arm_context(yhat_l: torch.Tensor, offsets) -> torch.Tensor:
    """[h, w] -> [h, w, N]: the value at each causal offset, 0 outside the grid."""
    r = max(max(-dy, abs(dx)) for dy, dx in offsets)
    h, w = yhat_l.shape
    p = F.pad(yhat_l, (r, r, r, 0))  # left, right, top, bottom
    return torch.stack([p[r + dy:r + dy + h, r + dx:r + dx + w] for dy, dx in offsets], -1)


def arm_mlp(ctx: torch.Tensor, P: dict, arch: Arch):
    """N-N-LinR x arm_layers, then N-2-Lin; returns (mu, s)."""
    h = ctx
    for i in range(arch.arm_layers):
        h = h + torch.relu(h @ P[f"arm.w{i}"].T + P[f"arm.b{i}"])
    out = h @ P["arm.wout"].T + P["arm.bout"]
    return out[..., 0], out[..., 1]


def laplace_cdf(x, mu, b):
    """Textbook Laplace CDF (used by the pins, not by the oracle's rate)."""
    z = (x - mu) / b
    return torch.where(z < 0, 0.5 * torch.exp(torch.clamp(z, max=0.0)),
                       1.0 - 0.5 * torch.exp(-torch.clamp(z, min=0.0)))


def laplace_bin_mass(yhat, mu, s):
    """P = F(yhat + 1/2) - F(yhat - 1/2) for the Laplace law of mean mu, scale exp(s).

    With d = yhat - mu both bounds lie on one side of mu when |d| >= 1/2, and then
    P = 1/2 exp(-(|d| - 1/2)/b) (1 - exp(-1/b)); otherwise
    P = 1 - 1/2 (exp(-(1/2 + d)/b) + exp(-(1/2 - d)/b)), written with expm1.  Each branch
    only sees arguments clamped to its own side, so neither can overflow.
    """
    b = torch.exp(torch.clamp(s, LOG_B_MIN, LOG_B_MAX))
    d = yhat - mu
    ad = torch.abs(d)
    ad_a = torch.clamp(ad, min=0.5)
    p_out = 0.5 * torch.exp(-(ad_a - 0.5) / b) * (-torch.expm1(-1.0 / b))
    d_b = torch.clamp(d, -0.5, 0.5)
    p_in = -0.5 * (torch.expm1(-(0.5 + d_b) / b) + torch.expm1(-(0.5 - d_b) / b))
    return torch.where(ad >= 0.5, p_out, p_in)


def rate_bits(yhat, mu, s):
    """-log2 p_psi(yhat) per latent, with the probability floored at 2^-16."""
    return -torch.log2(torch.clamp(laplace_bin_mass(yhat, mu, s), min=P_MIN))


def total_bits(yhat_levels, P, arch: Arch):
    offs = causal_offsets(arch.arm_ctx)
    bits = 0.0
    for yl in yhat_levels:
        mu, s = arm_mlp(arm_context(yl, offs), P, arch)
        bits = bits + rate_bits(yl, mu, s).sum()
    return bits


# --------------------------------------------------------------------------------------
# Upsampling f_upsilon (Table 1 "1-1-TConv-k", stride 2)
# --------------------------------------------------------------------------------------

def tconv2x_clamp(a: torch.Tensor, f: torch.Tensor, out_h: int, out_w: int) -> torch.Tensor:
    """One stride-2 transposed convolution, inputs read clamp-to-edge, output cropped.

    b[j] = sum over taps u with u = j + c (mod 2) of f[u] * a[clamp((j + c - u) / 2)],
    c = k/2 - 1, separately along rows and columns (f is a full k x k filter).
    """
    k = f.shape[-1]
    c = k // 2 - 1
    nh, nw = a.shape

    def taps_and_rows(phase, n_out, n_in):
        """Taps u of this output phase and, per tap, the clamped input index of each output."""
        j = np.arange(phase, n_out, 2)
        u = [t for t in range(k) if (phase + c - t) % 2 == 0]
        idx = np.stack([np.clip((j + c - t) // 2, 0, n_in - 1) for t in u])
        return u, torch.from_numpy(idx)

    rows = [taps_and_rows(ph, out_h, nh) for ph in (0, 1) if ph < out_h]
    cols = [taps_and_rows(pw, out_w, nw) for pw in (0, 1) if pw < out_w]
    b = a.new_zeros(out_h, out_w)
    for ph, (uy, iy) in enumerate(rows):
        for pw, (ux, ix) in enumerate(cols):
            # g[a, y, b, x] = input at (clamped row of tap uy[a] for output y, ... col ...)
            g = a.index_select(0, iy.reshape(-1)).index_select(1, ix.reshape(-1))
            g = g.reshape(len(uy), iy.shape[1], len(ux), ix.shape[1])
            b[ph::2, pw::2] = torch.einsum("aybx,ab->yx", g, f[uy][:, ux])
    return b


def upsample_level(yhat_l, f, l, shapes):
    """Level l brought to full resolution by l successive 2x steps with filter f."""
    a = yhat_l
    for j in range(l - 1, -1, -1):
        a = tconv2x_clamp(a, f, *shapes[j])
    return a


def upsample_all(yhat_levels, P, arch: Arch, shapes):
    feats = [yhat_levels[0]]
    for l in range(1, arch.levels):
        f = P[f"up.f{l}"] if arch.up_per_level else P["up.f"]
        feats.append(upsample_level(yhat_levels[l], f, l, shapes))
    return torch.stack(feats)


# --------------------------------------------------------------------------------------
# Synthesis f_theta (Table 1 "Synthesis")
# --------------------------------------------------------------------------------------

def conv3x3_replicate(h: torch.Tensor, w: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    return F.conv2d(F.pad(h[None], (1, 1, 1, 1), mode="replicate"), w, b)[0]


def synthesis(feat: torch.Tensor, P: dict, arch: Arch) -> torch.Tensor:
    """7-C-Conv-1 (ReLU), C-3-Conv-1 (ReLU), then 3-3-ConvR-3 layers (ReLU but the last)."""
    h = torch.relu(torch.einsum("ck,khw->chw", P["syn.wa"], feat) + P["syn.ba"][:, None, None])
    h = torch.relu(torch.einsum("ck,khw->chw", P["syn.wb"], h) + P["syn.bb"][:, None, None])
    for i in range(arch.syn_res3x3):
        z = conv3x3_replicate(h, P[f"syn.w3_{i}"], P[f"syn.b3_{i}"])
        h = h + (torch.relu(z) if i < arch.syn_res3x3 - 1 else z)
    return h


# --------------------------------------------------------------------------------------
# Loss, eq. (1)
# --------------------------------------------------------------------------------------

def forward(x, y_levels, P, arch: Arch, lam: float, u_levels=None, hard=False,
            soft_temp: float = 0.0):
    """Returns (loss, D, R_bpp, x_hat, y_hat levels).  x: [3, H, W] float64 in [0, 1]."""
    H, W = x.shape[1], x.shape[2]
    shapes = level_shapes(H, W, arch.levels)
    yhat = [quantize(y_levels[l], None if hard else u_levels[l], hard, soft_temp)
            for l in range(arch.levels)]
    R = total_bits(yhat, P, arch) / (H * W)
    xhat = synthesis(upsample_all(yhat, P, arch, shapes), P, arch)
    D = torch.mean((xhat - x) ** 2)
    return D + lam * R, D, R, xhat, yhat


@torch.no_grad()
def decision_margins(x, y_levels, P, arch: Arch, u_levels=None, hard=False, soft_temp=0.0):
    """Distance of every discrete decision of the forward pass to its tie.

    Where a decision sits within rounding error of its tie (a ReLU pre-activation near 0,
    a bin probability near the 2^-16 floor, a log-scale near a clamp bound), an FP32
    evaluation may legitimately take the other side, and the two one-sided derivatives
    differ.  Returns (arm, syn): per latent of each level, the smallest of |z| over the
    ARM's LinR pre-activations, |log2 P + 16| and the distance of s to its clamp bounds;
    per pixel, the smallest |pre-activation| of the synthesis ReLUs.
    """
    H, W = x.shape[1], x.shape[2]
    shapes = level_shapes(H, W, arch.levels)
    yhat = [torch.round(y) if hard else quantize(y, u, False, soft_temp) for y, u in
            zip(y_levels, u_levels if u_levels is not None else [None] * arch.levels)]
    offs = causal_offsets(arch.arm_ctx)
    arm = []
    for yl in yhat:
        h = arm_context(yl, offs)
        m = torch.full(yl.shape, float("inf"), dtype=DT)
        for i in range(arch.arm_layers):
            z = h @ P[f"arm.w{i}"].T + P[f"arm.b{i}"]
            m = torch.minimum(m, torch.min(torch.abs(z), -1).values)
            h = h + torch.relu(z)
        out = h @ P["arm.wout"].T + P["arm.bout"]
        mu, sc = out[..., 0], out[..., 1]
        pm = laplace_bin_mass(yl, mu, sc)
        m = torch.minimum(m, torch.abs(torch.log2(torch.clamp(pm, min=1e-300)) + 16.0))
        m = torch.minimum(m, torch.minimum(torch.abs(sc - LOG_B_MIN), torch.abs(sc - LOG_B_MAX)))
        arm.append(m.numpy())
    feat = upsample_all(yhat, P, arch, shapes)
    z = torch.einsum("ck,khw->chw", P["syn.wa"], feat) + P["syn.ba"][:, None, None]
    syn = torch.min(torch.abs(z), 0).values
    h = torch.relu(z)
    z = torch.einsum("ck,khw->chw", P["syn.wb"], h) + P["syn.bb"][:, None, None]
    syn = torch.minimum(syn, torch.min(torch.abs(z), 0).values)
    h = torch.relu(z)
    for i in range(arch.syn_res3x3 - 1):
        z = conv3x3_replicate(h, P[f"syn.w3_{i}"], P[f"syn.b3_{i}"])
        syn = torch.minimum(syn, torch.min(torch.abs(z), 0).values)
        h = h + torch.relu(z)
    return arm, syn.numpy()


def image_to_planar(rgb_hwc_u8: np.ndarray) -> torch.Tensor:
    """uint8 H x W x 3 -> float64 [3, H, W] with x = v / 255."""
    return torch.tensor(np.transpose(rgb_hwc_u8, (2, 0, 1)).astype(np.float64) / 255.0, dtype=DT)


class OracleEncoder:
    """Latents y, decoder parameters and Adam moments; one `step` is one iteration."""

    def __init__(self, rgb_hwc_u8: np.ndarray, arch: Arch, train: Train, init_params: dict):
        self.arch, self.train = arch, train
        self.x = image_to_planar(rgb_hwc_u8)
        self.H, self.W = self.x.shape[1], self.x.shape[2]
        self.shapes = level_shapes(self.H, self.W, arch.levels)
        self.y = [torch.zeros(h, w, dtype=DT, requires_grad=True) for h, w in self.shapes]
        self.P = params_from_numpy(init_params, arch)
        self.names = [n for n, _ in param_shapes(arch)]
        self.tensors = self.y + [self.P[n] for n in self.names]
        self.m = [torch.zeros_like(t) for t in self.tensors]
        self.v = [torch.zeros_like(t) for t in self.tensors]
        self.t = 0

    def noise(self, t: int):
        return [torch.tensor(u, dtype=DT)
                for u in philox.latent_noise(self.train.seed, t, self.shapes)]

    def is_hard(self, t: int) -> bool:
        return t >= self.train.ste_start

    def loss_and_grads(self, u_levels=None, hard=None):
        """Forward at the current iteration (its own noise unless given) and all gradients."""
        if hard is None:
            hard = self.is_hard(self.t)
        if u_levels is None and not hard:
            u_levels = self.noise(self.t)
        loss, D, R, _, _ = forward(self.x, self.y, self.P, self.arch, self.train.lam,
                                   u_levels, hard, self.train.soft_temp)
        grads = torch.autograd.grad(loss, self.tensors)
        return float(loss.detach()), float(D.detach()), float(R.detach()), [g.detach() for g in grads]

    def adam_update(self, grads):
        t = self.t + 1
        bc1 = 1.0 - ADAM_BETA1 ** t
        bc2 = 1.0 - ADAM_BETA2 ** t
        lr = self.train.lr
        with torch.no_grad():
            for p, g, m, v in zip(self.tensors, grads, self.m, self.v):
                m.mul_(ADAM_BETA1).add_((1.0 - ADAM_BETA1) * g)
                v.mul_(ADAM_BETA2).add_((1.0 - ADAM_BETA2) * g * g)
                p.sub_(lr * (m / bc1) / (torch.sqrt(v / bc2) + ADAM_EPS))
        self.t = t

    def step(self, u_levels=None):
        loss, D, R, grads = self.loss_and_grads(u_levels)
        self.adam_update(grads)
        return loss, D, R

    @torch.no_grad()
    def rd_cost(self, hard: bool = True):
        """(D, R_bpp, D + lambda R) with rint latents and no noise (or the current noise)."""
        u = None if hard else self.noise(self.t)
        loss, D, R, _, _ = forward(self.x, self.y, self.P, self.arch, self.train.lam, u, hard,
                                   self.train.soft_temp)
        return float(D), float(R), float(loss)

    @torch.no_grad()
    def decode(self) -> np.ndarray:
        """x_hat (H x W x 3, float64) from rint latents."""
        _, _, _, xhat, _ = forward(self.x, self.y, self.P, self.arch, self.train.lam, None, True)
        return xhat.permute(1, 2, 0).numpy().copy()

    def state_arrays(self):
        """y levels and parameters as float64 numpy arrays (by name for parameters)."""
        return ([t.detach().numpy().copy() for t in self.y],
                {n: self.P[n].detach().numpy().copy() for n in self.names})

    def set_latents(self, y_levels):
        with torch.no_grad():
            for t, a in zip(self.y, y_levels):
                t.copy_(torch.as_tensor(np.asarray(a, dtype=np.float64)))
