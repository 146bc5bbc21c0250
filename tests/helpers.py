"""Shared set-up for the parity tests: the same seeded inputs handed to the CUDA library
(through its C ABI binding) and to the FP64 oracle."""
from __future__ import annotations

import numpy as np
import torch

from oracle import coolchic as oc
from paper_2403_11651_gb300 import coolchic as cc
from paper_2403_11651_gb300 import synthetic as syn

ARCHS = {
    # name: (arm_ctx, arm_layers, up_kernel, up_per_level, syn_hidden, syn_res3x3)
    "c1": (8, 2, 8, 1, 8, 2),
    "c2": (24, 2, 8, 1, 40, 2),
    "t300": (8, 1, 4, 0, 8, 1),
    "t545": (8, 2, 4, 0, 16, 2),
    "t1079": (16, 2, 4, 0, 16, 2),
}


def config_dict(arch: str, lam=1e-3, lr=1e-2, total_iters=100, ste_frac=0.0, soft_temp=0.0):
    n, nl, k, pl, c, nr = ARCHS[arch]
    return dict(levels=7, arm_ctx=n, arm_layers=nl, up_kernel=k, up_per_level=bool(pl),
                syn_hidden=c, syn_res3x3=nr, lam=lam, lr=lr, total_iters=total_iters,
                ste_frac=ste_frac, soft_temp=soft_temp)


def oracle_arch(d: dict) -> oc.Arch:
    return oc.Arch(levels=7, arm_ctx=d["arm_ctx"], arm_layers=d["arm_layers"],
                   up_kernel=d["up_kernel"], up_per_level=bool(d["up_per_level"]),
                   syn_hidden=d["syn_hidden"], syn_res3x3=d["syn_res3x3"])


class Pair:
    """A CUDA context and an oracle encoder built from identical inputs."""

    def __init__(self, d: dict, H: int, W: int, seed: int = 0, random_state: bool = False,
                 state_scale: float = 1.5):
        self.d, self.H, self.W, self.seed = d, H, W, seed
        self.cfg = cc.make_config(d, seed=seed)
        self.rgb = syn.synthetic_image(H, W, seed)
        self.init = syn.initial_parameters(syn.ArchSizes.from_config(d), seed)
        rng = np.random.default_rng(seed + 1000)
        if random_state:
            for k in self.init:   # non-zero biases so every gradient term is exercised
                if ".b" in k:
                    self.init[k] = rng.uniform(-0.1, 0.1, self.init[k].shape).astype(np.float32)
        self.flat_init = cc.flatten_params(self.init, self.cfg)
        self.n_params = cc.cc_param_count(self.cfg)
        self.n_lat = cc.cc_latent_count(self.cfg, H, W)
        self.ctx = cc.cc_init_image(self.cfg, self.rgb, H, W, self.flat_init)
        self.oracle = oc.OracleEncoder(
            self.rgb, oracle_arch(d),
            oc.Train(lam=d["lam"], lr=d["lr"], total_iters=d["total_iters"],
                     ste_frac=d["ste_frac"], seed=seed, soft_temp=d.get("soft_temp", 0.0)),
            self.init)
        if random_state:
            y = [rng.normal(0, state_scale, s).astype(np.float32) for s in cc.level_shapes(H, W)]
            self.set_latents(y)

    def set_latents(self, levels):
        flat = np.concatenate([np.asarray(a, np.float32).ravel() for a in levels])
        cc.cc_set_latents(self.ctx, flat)
        self.oracle.set_latents([a.astype(np.float64) for a in levels])

    def gpu_grads(self, noise_levels=None, hard=-1):
        noise = None
        if noise_levels is not None:
            noise = np.concatenate([np.asarray(a, np.float32).ravel() for a in noise_levels])
        g, D, R = cc.cc_forward_backward(self.ctx, self.n_lat + self.n_params, noise, hard)
        return (cc.split_latents(g[:self.n_lat], self.H, self.W),
                cc.unflatten_params(g[self.n_lat:], self.cfg), D, R)

    def oracle_grads(self, noise_levels=None, hard=False):
        u = None
        if noise_levels is not None:
            u = [torch.tensor(np.asarray(a, np.float64)) for a in noise_levels]
        loss, D, R, grads = self.oracle.loss_and_grads(u_levels=u, hard=hard)
        gy = [g.numpy() for g in grads[:7]]
        gp = {n: g.numpy() for n, g in zip(self.oracle.names, grads[7:])}
        return gy, gp, D, R

    def close(self):
        cc.cc_free(self.ctx)
        self.ctx = None


def assert_group_close(got, ref, rtol, name=""):
    """max |got - ref| <= rtol * max |ref| over the group (scale-relative)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = float(np.max(np.abs(ref))) if ref.size else 0.0
    err = float(np.max(np.abs(got - ref))) if ref.size else 0.0
    if err > rtol * max(scale, 1e-30):
        bad = np.abs(got - ref) > rtol * scale
        idx = np.argsort(-np.abs(got - ref).ravel())[:5]
        worst = [(np.unravel_index(i, ref.shape), float(got.ravel()[i]), float(ref.ravel()[i]))
                 for i in idx]
        raise AssertionError(f"{name}: max err {err:.3e} vs scale {scale:.3e}; "
                             f"{int(bad.sum())} of {bad.size} beyond tolerance; worst {worst}")


def margins(pair, noise_levels=None, hard=False):
    """The oracle's decision margins for the pair's current state."""
    enc = pair.oracle
    u = None if noise_levels is None else [torch.tensor(np.asarray(a, np.float64))
                                           for a in noise_levels]
    return oc.decision_margins(enc.x, [t.detach() for t in enc.y],
                               {k: v.detach() for k, v in enc.P.items()}, enc.arch, u, hard,
                               enc.train.soft_temp)


def assert_latents_close_with_ties(got, ref, level, arm_margin, syn_margin, offsets, rtol,
                                   delta=1e-5, max_outliers=None):
    """Element-wise tolerance on one latent level, except at latents whose gradient depends
    on a decision within `delta` of its tie in the oracle (an ARM decision of the latent
    itself or of a latent whose context holds it, or a synthesis ReLU in its pixel
    footprint).  Such exemptions must stay rare: at most max_outliers (default
    max(4, 1e-4 of the level)); one ARM tie reaches the latent and the N latents whose
    context holds it."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = float(np.max(np.abs(ref)))
    bad = np.argwhere(np.abs(got - ref) > rtol * scale)
    cap = max(4, 1e-4 * ref.size) if max_outliers is None else max_outliers
    assert len(bad) <= cap, f"level {level}: {len(bad)} outliers"
    h, w = ref.shape
    Hp, Wp = syn_margin.shape
    for r, c in bad:
        ok = False
        for dy, dx in [(0, 0)] + [(-a, -b) for a, b in offsets]:
            pr, pc = r + dy, c + dx
            if 0 <= pr < h and 0 <= pc < w and arm_margin[pr, pc] < delta:
                ok = True
        s = 1 << level
        y0, y1 = max(0, (r - 4) * s - 2), min(Hp, (r + 5) * s + 2)
        x0, x1 = max(0, (c - 4) * s - 2), min(Wp, (c + 5) * s + 2)
        if np.min(syn_margin[y0:y1, x0:x1]) < delta:
            ok = True
        assert ok, (f"level {level} ({r},{c}): {got[r, c]:.6e} vs {ref[r, c]:.6e} "
                    f"(scale {scale:.3e}) with no near-tie decision nearby")


STATE_MAGIC, STATE_VERSION = 0x31534343, 1   # "CCS1", the header of cc_get_state


def state_blob(d: dict, H: int, W: int, seed: int, iteration: int, y_flat, p_flat,
               my, vy, mp, vp) -> bytes:
    """A cc_set_state blob (include/coolchic.h) from float32 arrays in flat orders: the
    header (magic, version, H, W, latent and parameter counts, iteration, seed, the
    architecture fields), then y, parameters, latent m, latent v, parameter m, parameter v."""
    import struct
    arrays = [np.asarray(a, np.float32).ravel() for a in (y_flat, p_flat, my, vy, mp, vp)]
    arch = [d["arm_ctx"], d["arm_layers"], d["up_kernel"], int(d["up_per_level"]),
            d["syn_hidden"], d["syn_res3x3"], 7, 0]
    hdr = struct.pack("<IIiiiiiiQ8i", STATE_MAGIC, STATE_VERSION, H, W, arrays[0].size,
                      arrays[1].size, iteration, 0, seed & 0xFFFFFFFFFFFFFFFF, *arch)
    return hdr + b"".join(a.tobytes() for a in arrays)


def share_oracle_state(pair: Pair):
    """Round the oracle's whole state (latents, parameters, Adam moments) to float32, put
    the rounded values back into the oracle and load them into the CUDA context, so that
    both continue from one identical state at the oracle's iteration."""
    enc = pair.oracle
    nl = len(enc.y)

    def flat(ts):
        return np.concatenate([np.asarray(t.detach().numpy(), np.float32).ravel() for t in ts])

    parts = [flat(enc.tensors[:nl]), flat(enc.tensors[nl:]), flat(enc.m[:nl]), flat(enc.v[:nl]),
             flat(enc.m[nl:]), flat(enc.v[nl:])]
    with torch.no_grad():
        for group, src in ((enc.tensors, parts[0:2]), (enc.m, parts[2:3] + parts[4:5]),
                           (enc.v, parts[3:4] + parts[5:6])):
            vals = np.concatenate(src)
            k = 0
            for t in group:
                n = t.numel()
                t.copy_(torch.from_numpy(vals[k:k + n].astype(np.float64)).reshape(t.shape))
                k += n
    blob = state_blob(pair.d, pair.H, pair.W, pair.seed, enc.t, *parts)
    cc.cc_set_state(pair.ctx, blob)
