"""Seeded synthetic inputs shared by the CUDA path's tests, the bench and the oracle's tests.

This module holds no arithmetic of the coding method itself: it only draws inputs.

* ``synthetic_image``: an RGB uint8 image standing in for the Kodak / CLIC-pro images the
  paper evaluates on (Sec. I, Fig. 1, Fig. 3): a 1/f^2 Gaussian random field shared by the
  three channels plus weaker per-channel fields, twenty constant-colour polygons and 5 %
  Gaussian texture noise, clipped and quantised to 8 bits.
* ``initial_parameters``: the starting value of every decoder parameter, by name.  Weights
  are uniform in +-1/sqrt(fan_in), biases zero, and each 2x upsampling filter starts as the
  2x resampling filter of Keys' cubic kernel (a = -0.75) for k = 8, or the bilinear one for
  k = 4, so that every polyphase component sums to one.
* ``uniform_noise``: explicit quantisation noise in [-1/2, 1/2) on a 2^-24 grid, for the
  tests that pass noise in instead of drawing it from the counter-based generator.
* ``synthetic_latents``: an integer latent pyramid for the bitstream benchmarks: level l
  draws rounded Laplace values of scale 0.4 + 0.6 l (coarser levels carry larger values,
  as in trained Cool-chic pyramids).

Every value is exactly representable in float32, so both implementations start from
bit-identical inputs.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "ArchSizes",
    "level_shapes",
    "synthetic_image",
    "initial_parameters",
    "uniform_noise",
    "synthetic_latents",
    "warm_initial_parameters",
    "keys_cubic",
]


class ArchSizes:
    """Sizes of the decoder networks (Table 1 notation), enough to shape the initial values."""

    def __init__(self, arm_ctx=24, arm_layers=2, up_kernel=8, up_per_level=True,
                 syn_hidden=40, syn_res3x3=2, levels=7):
        self.arm_ctx = int(arm_ctx)
        self.arm_layers = int(arm_layers)
        self.up_kernel = int(up_kernel)
        self.up_per_level = bool(up_per_level)
        self.syn_hidden = int(syn_hidden)
        self.syn_res3x3 = int(syn_res3x3)
        self.levels = int(levels)

    @classmethod
    def from_config(cls, cfg: dict) -> "ArchSizes":
        return cls(arm_ctx=cfg["arm_ctx"], arm_layers=cfg["arm_layers"],
                   up_kernel=cfg["up_kernel"], up_per_level=cfg["up_per_level"],
                   syn_hidden=cfg["syn_hidden"], syn_res3x3=cfg["syn_res3x3"],
                   levels=cfg.get("levels", 7))


def level_shapes(H: int, W: int, levels: int = 7):
    """Grid size of each latent level: ceil(H / 2^l) x ceil(W / 2^l)."""
    return [(-(-H // (1 << l)), -(-W // (1 << l))) for l in range(levels)]


def _grf(rng: np.random.Generator, H: int, W: int) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian field with amplitude spectrum 1/|f| (power 1/f^2)."""
    white = rng.standard_normal((H, W))
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    f = np.sqrt(fy * fy + fx * fx)
    amp = np.zeros_like(f)
    amp[f > 0] = 1.0 / f[f > 0]
    field = np.real(np.fft.ifft2(np.fft.fft2(white) * amp))
    field -= field.mean()
    sd = field.std()
    return field / sd if sd > 0 else field


def _polygon_mask(H: int, W: int, vx: np.ndarray, vy: np.ndarray) -> np.ndarray:
    """Even-odd rule over pixel centres."""
    py = (np.arange(H) + 0.5)[:, None]
    px = (np.arange(W) + 0.5)[None, :]
    inside = np.zeros((H, W), dtype=bool)
    n = len(vx)
    for i in range(n):
        x1, y1 = vx[i], vy[i]
        x2, y2 = vx[(i + 1) % n], vy[(i + 1) % n]
        if y1 == y2:
            continue
        crosses = (y1 > py) != (y2 > py)
        xint = (x2 - x1) * (py - y1) / (y2 - y1) + x1
        inside ^= crosses & (px < xint)
    return inside


def synthetic_image(H: int, W: int, seed: int, n_polygons: int = 20,
                    noise_sigma: float = 0.05) -> np.ndarray:
    """Seeded H x W x 3 uint8 image (row-major, channels last)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lum = _grf(rng, H, W)
    img = np.stack([lum + 0.3 * _grf(rng, H, W) for _ in range(3)], axis=-1)
    sd = img.std()
    img = 0.5 + 0.2 * (img - img.mean()) / (sd if sd > 0 else 1.0)
    for _ in range(n_polygons):
        nv = int(rng.integers(3, 9))
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        r = rng.uniform(0.03, 0.2) * min(H, W)
        ang = np.sort(rng.uniform(0.0, 2.0 * math.pi, nv))
        rad = r * rng.uniform(0.5, 1.0, nv)
        mask = _polygon_mask(H, W, cx + rad * np.cos(ang), cy + rad * np.sin(ang))
        img[mask] = rng.uniform(0.0, 1.0, 3)
    img = img + rng.normal(0.0, noise_sigma, img.shape)
    return np.clip(np.rint(img * 255.0), 0, 255).astype(np.uint8)


def keys_cubic(x: float, a: float = -0.75) -> float:
    """Keys' cubic convolution kernel."""
    x = abs(x)
    if x <= 1.0:
        return (a + 2.0) * x ** 3 - (a + 3.0) * x ** 2 + 1.0
    if x < 2.0:
        return a * x ** 3 - 5.0 * a * x ** 2 + 8.0 * a * x - 4.0 * a
    return 0.0


def _resampling_filter_1d(k: int) -> np.ndarray:
    """Taps of a 2x resampler at output phases +-1/4, laid out for a k-tap transposed conv."""
    if k == 8:
        half = [keys_cubic(d) for d in (1.75, 1.25, 0.75, 0.25)]
    elif k == 4:
        half = [0.25, 0.75]  # linear interpolation at distances 3/4 and 1/4
    else:
        raise ValueError(f"unsupported upsampling kernel size {k}")
    return np.array(half + half[::-1], dtype=np.float64)


def initial_parameters(arch: ArchSizes, seed: int) -> dict:
    """Named float32 arrays with the starting decoder parameters."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5EED1234))
    out = {}

    def uni(shape, fan_in):
        bound = 1.0 / math.sqrt(fan_in)
        return rng.uniform(-bound, bound, shape).astype(np.float32)

    n = arch.arm_ctx
    for i in range(arch.arm_layers):
        out[f"arm.w{i}"] = uni((n, n), n)
        out[f"arm.b{i}"] = np.zeros(n, np.float32)
    out["arm.wout"] = uni((2, n), n)
    out["arm.bout"] = np.zeros(2, np.float32)
    f1 = _resampling_filter_1d(arch.up_kernel)
    f2 = np.outer(f1, f1).astype(np.float32)
    if arch.up_per_level:
        for l in range(1, arch.levels):
            out[f"up.f{l}"] = f2.copy()
    else:
        out["up.f"] = f2.copy()
    c = arch.syn_hidden
    out["syn.wa"] = uni((c, arch.levels), arch.levels)
    out["syn.ba"] = np.zeros(c, np.float32)
    out["syn.wb"] = uni((3, c), c)
    out["syn.bb"] = np.zeros(3, np.float32)
    for i in range(arch.syn_res3x3):
        out[f"syn.w3_{i}"] = uni((3, 3, 3, 3), 27)
        out[f"syn.b3_{i}"] = np.zeros(3, np.float32)
    return out


def uniform_noise(H: int, W: int, seed: int, levels: int = 7):
    """Per-level float32 noise in [-1/2, 1/2), each value a multiple of 2^-24."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0xA5A5A5))
    out = []
    for (h, w) in level_shapes(H, W, levels):
        k = rng.integers(0, 1 << 24, size=(h, w), dtype=np.int64)
        out.append((k.astype(np.float64) * 2.0 ** -24 - 0.5).astype(np.float32))
    return out


def synthetic_latents(H: int, W: int, seed: int, levels: int = 7):
    """Per-level int32 planes of rounded Laplace values, scale 0.4 + 0.6 l at level l."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5A5A5A))
    return [np.rint(rng.laplace(0.0, 0.4 + 0.6 * l, size=s)).astype(np.int32)
            for l, s in enumerate(level_shapes(H, W, levels))]


def warm_initial_parameters(seed: int) -> np.ndarray:
    """Flat float32 parameters of the warm-start predictor: weights uniform in
    +-1/sqrt(fan_in), biases 0 (layer order of include/coolchic.h)."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x3C3C3C))
    shapes = ([((32, 3, 3, 3), 27), ((32,), 0)]
              + [s for _ in range(3) for s in (((32, 32, 3, 3), 288), ((32,), 0))]
              + [s for _ in range(4) for s in (((1, 32, 1, 1), 32), ((1,), 0))]
              + [((1, 3, 3, 3), 27), ((1,), 0)])
    out = []
    for shape, fan_in in shapes:
        n = int(np.prod(shape))
        if fan_in:
            b = 1.0 / math.sqrt(fan_in)
            out.append(rng.uniform(-b, b, n).astype(np.float32))
        else:
            out.append(np.zeros(n, np.float32))
    return np.concatenate(out)
