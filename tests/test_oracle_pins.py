"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: numbers printed in the
paper (Table 1, Fig. 5 via eq. (2)), closed forms, library routines (numpy's Philox,
scipy's Laplace law, torch's bicubic resampling), invariants, and brute-force loops written
straight from the definitions on tiny inputs.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import coolchic as oc
from oracle import philox
from paper_2403_11651_gb300 import synthetic as syn

DT = torch.float64


def _arch_row(row, per_level=False):
    return oc.Arch(arm_ctx=row["arm_ctx"], arm_layers=row["arm_layers"],
                   up_kernel=row["up_kernel"], up_per_level=per_level,
                   syn_hidden=row["syn_hidden"], syn_res3x3=row["syn_res3x3"])


@pytest.fixture(scope="module")
def golden(golden_dir):
    with open(os.path.join(golden_dir, "table1_fig5.json")) as f:
        return json.load(f)


# ---------------------------------------------------------------- architecture (Table 1)

def test_table1_parameter_counts(golden):
    """Table 1: 281 / 525 / 941 / 1925 parameters with one shared upsampling filter."""
    for row in golden["table1"]:
        assert oc.param_count(_arch_row(row)) == row["params"], row


def test_fig5_mac_per_pixel(golden):
    """Fig. 5 x-coordinates / (3 N) (eq. (2)) give kappa_dec = 299 / 545.3 / 1079 / 2291."""
    iters = {102950, 12950, 10600, 3600, 1600, 1100, 600}
    for row in golden["table1"]:
        pts = golden["fig5"][str(row["mac"])]
        kappa = pts[0] / (3 * 102950)
        for p in pts:  # every point of the curve is 3 N kappa with a plausible N
            n = p / (3 * kappa)
            assert abs(n - round(n)) < 1e-6 and round(n) in iters
        mac = oc.macs_per_pixel(_arch_row(row))["total"]
        assert abs(mac - kappa) / kappa < 5e-3, (row["mac"], mac, kappa)
        assert abs(mac - row["mac"]) / row["mac"] < 1e-2


def test_arm_dominates_macs(golden):
    """Sec. III-A: most of the complexity is the ARM's (about 70 % at 2300 MAC)."""
    row = golden["table1"][3]
    m = oc.macs_per_pixel(_arch_row(row))
    assert m["arm"] > m["synthesis"] > m["upsampling"]
    assert 0.65 < m["arm"] / m["total"] < 0.75


def test_causal_offsets():
    o8 = oc.causal_offsets(8)
    assert o8 == [(-2, 0), (-1, -2), (-1, -1), (-1, 0), (-1, 1), (-1, 2), (0, -2), (0, -1)]
    o24 = oc.causal_offsets(24)
    ball = sorted((dy, dx) for dy in range(-4, 1) for dx in range(-4, 5)
                  if (dy < 0 or dx < 0) and dy * dy + dx * dx <= 16)
    assert o24 == ball and len(ball) == 24
    for dy, dx in oc.causal_offsets(16):
        assert dy < 0 or (dy == 0 and dx < 0)


def test_level_shapes_odd():
    assert oc.level_shapes(1080, 1920)[3] == (135, 240)
    assert oc.level_shapes(1080, 1920)[4] == (68, 120)
    assert oc.level_shapes(67, 45)[6] == (2, 1)


# ---------------------------------------------------------------- Laplace rate (eq. (1))

def _bins(mu, s, k):
    return oc.laplace_bin_mass(torch.tensor(k, dtype=DT), torch.tensor(mu, dtype=DT),
                               torch.tensor(s, dtype=DT))


def test_laplace_bins_sum_to_one():
    rng = np.random.default_rng(1)
    for _ in range(40):
        mu = rng.uniform(-20, 20)
        s = rng.uniform(oc.LOG_B_MIN, math.log(50.0))
        b = math.exp(s)
        k = np.arange(math.floor(mu - 60 * b) - 1, math.ceil(mu + 60 * b) + 2, dtype=np.float64)
        assert abs(float(_bins(mu, s, k).sum()) - 1.0) < 1e-12


def test_laplace_closed_form_mu0():
    """mu = 0: P(0) = 1 - exp(-1/(2b)) and P(k) = exp(-|k|/b) sinh(1/(2b)) for k != 0."""
    for b in (0.05, 0.3, 1.0, 4.0, 100.0):
        k = np.arange(-30, 31, dtype=np.float64)
        p = _bins(0.0, math.log(b), k).numpy()
        ref = np.where(k == 0, 1 - math.exp(-0.5 / b), np.exp(-np.abs(k) / b) * math.sinh(0.5 / b))
        np.testing.assert_allclose(p, ref, rtol=1e-12, atol=1e-300)


def test_laplace_matches_scipy():
    from scipy.stats import laplace
    rng = np.random.default_rng(2)
    mu = rng.uniform(-3, 3, 500)
    b = np.exp(rng.uniform(math.log(0.2), math.log(5.0), 500))
    y = np.round(rng.uniform(-6, 6, 500)) + rng.uniform(-0.5, 0.5, 500)
    ref = laplace.cdf(y + 0.5, mu, b) - laplace.cdf(y - 0.5, mu, b)
    p = oc.laplace_bin_mass(torch.tensor(y), torch.tensor(mu), torch.tensor(np.log(b))).numpy()
    keep = ref > 1e-6
    np.testing.assert_allclose(p[keep], ref[keep], rtol=1e-9)


def test_rate_floor_and_scale_clamp():
    y = torch.tensor([40.0], dtype=DT, requires_grad=True)
    mu = torch.tensor([0.0], dtype=DT, requires_grad=True)
    s = torch.tensor([0.0], dtype=DT, requires_grad=True)
    r = oc.rate_bits(y, mu, s)
    assert float(r.detach()) == 16.0
    r.sum().backward()
    assert float(y.grad) == 0 and float(mu.grad) == 0 and float(s.grad) == 0
    # scale clamp: s far outside the range has no gradient
    s2 = torch.tensor([30.0], dtype=DT, requires_grad=True)
    oc.rate_bits(torch.tensor([0.2], dtype=DT), torch.tensor([0.0], dtype=DT), s2).sum().backward()
    assert float(s2.grad) == 0


# ---------------------------------------------------------------- ARM

def _arm_params(n, layers, seed):
    a = syn.ArchSizes(arm_ctx=n, arm_layers=layers)
    p = syn.initial_parameters(a, seed)
    rng = np.random.default_rng(seed)
    for i in range(layers):
        p[f"arm.b{i}"] = rng.uniform(-0.3, 0.3, n).astype(np.float32)
    p["arm.bout"] = np.array([0.1, -0.2], np.float32)
    return {k: torch.tensor(v.astype(np.float64)) for k, v in p.items() if k.startswith("arm")}


def test_arm_bruteforce_tiny():
    """Per-latent loops straight from the definition, textbook CDF difference."""
    n, layers = 8, 2
    arch = oc.Arch(arm_ctx=n, arm_layers=layers)
    P = _arm_params(n, layers, 3)
    rng = np.random.default_rng(4)
    yh = rng.normal(0, 1.5, (5, 6))
    yt = torch.tensor(yh)
    mu, s = oc.arm_mlp(oc.arm_context(yt, oc.causal_offsets(n)), P, arch)
    bits = oc.rate_bits(yt, mu, s).numpy()
    Wn = {k: v.numpy() for k, v in P.items()}
    for r in range(5):
        for c in range(6):
            ctx = np.array([yh[r + dy, c + dx] if (0 <= r + dy and 0 <= c + dx < 6) else 0.0
                            for dy, dx in oc.causal_offsets(n)])
            h = ctx
            for i in range(layers):
                h = h + np.maximum(Wn[f"arm.w{i}"] @ h + Wn[f"arm.b{i}"], 0.0)
            m_, s_ = Wn["arm.wout"] @ h + Wn["arm.bout"]
            b = math.exp(min(max(s_, math.log(1e-2)), math.log(1e3)))

            def cdf(x):
                return 0.5 * math.exp((x - m_) / b) if x < m_ else 1 - 0.5 * math.exp(-(x - m_) / b)
            p = max(cdf(yh[r, c] + 0.5) - cdf(yh[r, c] - 0.5), 2.0 ** -16)
            assert abs(bits[r, c] + math.log2(p)) < 1e-9 * max(1.0, abs(math.log2(p)))


def test_arm_causality():
    """Bits of latent p change with its context and never with later latents or other levels."""
    n = 24
    arch = oc.Arch(arm_ctx=n)
    P = _arm_params(n, 2, 5)
    rng = np.random.default_rng(6)
    base = rng.normal(0, 1, (9, 11))

    def bits_of(y):
        t = torch.tensor(y)
        mu, s = oc.arm_mlp(oc.arm_context(t, oc.causal_offsets(n)), P, arch)
        return oc.rate_bits(t, mu, s).numpy()

    b0 = bits_of(base)
    p = (5, 5)
    for q in [(5, 6), (5, 10), (6, 0), (8, 10), (6, 5)]:   # raster-later positions
        y = base.copy()
        y[q] += 3.7
        b1 = bits_of(y)
        assert b1[p] == b0[p]
        # every latent raster-before q is unchanged
        flat = np.arange(base.size).reshape(base.shape)
        before = flat < flat[q]
        assert np.array_equal(b1[before], b0[before])
    for dy, dx in oc.causal_offsets(n):
        y = base.copy()
        y[p[0] + dy, p[1] + dx] += 3.7
        assert bits_of(y)[p] != b0[p]


# ---------------------------------------------------------------- upsampling

def _tconv_loops(a, f, m_h, m_w):
    """b[j] = sum over all (virtual) inputs i of a[clamp(i)] f[j - 2i + c], 0 <= j-2i+c < k."""
    k = f.shape[0]
    c = k // 2 - 1
    nh, nw = a.shape
    out = np.zeros((m_h, m_w))
    for jy in range(m_h):
        for jx in range(m_w):
            acc = 0.0
            for iy in range(-k, nh + k):
                uy = jy - 2 * iy + c
                if not 0 <= uy < k:
                    continue
                for ix in range(-k, nw + k):
                    ux = jx - 2 * ix + c
                    if not 0 <= ux < k:
                        continue
                    acc += a[min(max(iy, 0), nh - 1), min(max(ix, 0), nw - 1)] * f[uy, ux]
            out[jy, jx] = acc
    return out


@pytest.mark.parametrize("k,shape,out", [(8, (4, 5), (8, 10)), (8, (3, 4), (5, 7)),
                                          (4, (3, 3), (6, 5)), (8, (1, 1), (1, 2)),
                                          (8, (2, 1), (3, 1))])
def test_tconv_bruteforce(k, shape, out):
    rng = np.random.default_rng(7)
    a = rng.normal(size=shape)
    f = rng.normal(size=(k, k))
    got = oc.tconv2x_clamp(torch.tensor(a), torch.tensor(f), *out).numpy()
    np.testing.assert_allclose(got, _tconv_loops(a, f, *out), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("H,W", [(64, 64), (67, 45), (13, 200)])
def test_upsampling_constant_field_exact(H, W):
    """With the resampling init every phase sums to 1: constants are reproduced, borders too."""
    arch = oc.Arch()
    P = {k: torch.tensor(v.astype(np.float64))
         for k, v in syn.initial_parameters(syn.ArchSizes(), 0).items()}
    shapes = oc.level_shapes(H, W)
    y = [torch.full(s, 0.37 * (l + 1), dtype=DT) for l, s in enumerate(shapes)]
    feats = oc.upsample_all(y, P, arch, shapes)
    for l in range(7):
        assert torch.max(torch.abs(feats[l] - 0.37 * (l + 1))) < 1e-12


def test_upsampling_step_is_bicubic_resampling():
    """Keys-cubic init: one step equals torch's bicubic 2x resize (align_corners=False)."""
    f1 = np.array([syn.keys_cubic(d) for d in (1.75, 1.25, 0.75, 0.25, 0.25, 0.75, 1.25, 1.75)])
    f = torch.tensor(np.outer(f1, f1))
    a = torch.tensor(np.random.default_rng(8).normal(size=(9, 13)))
    ref = torch.nn.functional.interpolate(a[None, None], scale_factor=2, mode="bicubic",
                                          align_corners=False)[0, 0]
    got = oc.tconv2x_clamp(a, f, 18, 26)
    assert torch.max(torch.abs(got - ref)) < 1e-12


# ---------------------------------------------------------------- synthesis

def _syn_loops(feat, P, arch):
    C, H, W = feat.shape
    Pn = {k: v.numpy() for k, v in P.items()}
    h = np.zeros((3, H, W))
    for y in range(H):
        for x in range(W):
            z1 = np.maximum(Pn["syn.wa"] @ feat[:, y, x] + Pn["syn.ba"], 0)
            h[:, y, x] = np.maximum(Pn["syn.wb"] @ z1 + Pn["syn.bb"], 0)
    for i in range(arch.syn_res3x3):
        w, b = Pn[f"syn.w3_{i}"], Pn[f"syn.b3_{i}"]
        nh = h.copy()
        for y in range(H):
            for x in range(W):
                z = b.copy()
                for o in range(3):
                    for ci in range(3):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                yy = min(max(y + dy, 0), H - 1)
                                xx = min(max(x + dx, 0), W - 1)
                                z[o] += w[o, ci, dy + 1, dx + 1] * h[ci, yy, xx]
                nh[:, y, x] = h[:, y, x] + (np.maximum(z, 0) if i < arch.syn_res3x3 - 1 else z)
        h = nh
    return h


def test_synthesis_bruteforce():
    arch = oc.Arch(syn_hidden=8)
    rng = np.random.default_rng(9)
    named = syn.initial_parameters(syn.ArchSizes(syn_hidden=8), 1)
    P = {k: torch.tensor(v.astype(np.float64) + (rng.uniform(-.2, .2, v.shape) if "b" in k.split(".")[1][:1] else 0))
         for k, v in named.items()}
    feat = rng.normal(size=(7, 5, 6))
    got = oc.synthesis(torch.tensor(feat), P, arch).numpy()
    np.testing.assert_allclose(got, _syn_loops(feat, P, arch), rtol=1e-12, atol=1e-12)


def test_synthesis_zero_weights_constant():
    arch = oc.Arch(syn_hidden=8)
    named = syn.initial_parameters(syn.ArchSizes(syn_hidden=8), 1)
    P = {k: torch.zeros(v.shape, dtype=DT) for k, v in named.items()}
    P["syn.bb"] = torch.tensor([0.2, 0.4, 0.6], dtype=DT)
    P["syn.b3_1"] = torch.tensor([0.1, -0.1, 0.05], dtype=DT)
    feat = torch.randn(7, 6, 7, dtype=DT)
    out = oc.synthesis(feat, P, arch)
    for c, v in enumerate([0.3, 0.3, 0.65]):
        assert torch.max(torch.abs(out[c] - v)) < 1e-15


# ---------------------------------------------------------------- quantisation, noise, loss

def test_ste_forward_rint_backward_identity():
    y = torch.tensor([0.5, 1.5, -0.5, 2.49, -2.51, 0.0], dtype=DT, requires_grad=True)
    q = oc.quantize(y, None, True)
    assert q.tolist() == [0.0, 2.0, -0.0, 2.0, -3.0, 0.0]
    (q * torch.arange(6, dtype=DT)).sum().backward()
    assert y.grad.tolist() == [0, 1, 2, 3, 4, 5]


def test_noise_statistics():
    u = np.concatenate([a.ravel() for a in philox.latent_noise(11, 3, [(1000, 1000)])])
    assert u.min() >= -0.5 and u.max() < 0.5
    n = u.size
    assert abs(u.mean()) < 4 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 2e-3
    assert np.all(np.round(u * 2 ** 24) == u * 2 ** 24)
    u2 = philox.latent_noise(11, 4, [(1000, 1000)])[0].ravel()
    assert abs(np.corrcoef(u, u2)[0, 1]) < 5e-3


def test_philox_matches_numpy_philox4x64():
    """numpy's Philox is Philox4x64-10 and generates from counter + 1."""
    rng = np.random.default_rng(12)
    for _ in range(20):
        ctr = [int(v) for v in rng.integers(0, 2 ** 63, 4)]
        key = [int(v) for v in rng.integers(0, 2 ** 63, 2)]
        g = np.random.Philox(counter=np.array(ctr, np.uint64), key=np.array(key, np.uint64))
        raw = [int(v) for v in g.random_raw(4)]
        assert raw == philox.philox4_reference([ctr[0] + 1] + ctr[1:], key, width=64)


def test_philox32_vectorised_matches_reference():
    rng = np.random.default_rng(13)
    ctr = rng.integers(0, 2 ** 32, (200, 4), dtype=np.uint64)
    key = (0xDEADBEEF, 0x12345678)
    got = philox.philox4x32_10(ctr, key)
    for i in range(200):
        assert [int(v) for v in got[i]] == philox.philox4_reference(ctr[i], key, 32)


def test_distortion_is_mse():
    rgb = syn.synthetic_image(8, 10, 1)
    x = oc.image_to_planar(rgb)
    assert x.shape == (3, 8, 10) and float(x.max()) <= 1.0
    np.testing.assert_allclose(x[1, 3, 4].item(), rgb[3, 4, 1] / 255.0, rtol=0, atol=0)


# ---------------------------------------------------------------- gradients and Adam

def _small_encoder(arch, H=12, W=10, lam=1e-2, seed=0):
    sizes = syn.ArchSizes(arm_ctx=arch.arm_ctx, arm_layers=arch.arm_layers,
                          up_kernel=arch.up_kernel, up_per_level=arch.up_per_level,
                          syn_hidden=arch.syn_hidden, syn_res3x3=arch.syn_res3x3)
    init = syn.initial_parameters(sizes, seed)
    rng = np.random.default_rng(seed + 100)
    for k in init:  # non-zero biases so every term has a gradient
        if ".b" in k:
            init[k] = rng.uniform(-0.1, 0.1, init[k].shape).astype(np.float32)
    enc = oc.OracleEncoder(syn.synthetic_image(H, W, seed), arch,
                           oc.Train(lam=lam, total_iters=100), init)
    enc.set_latents([rng.normal(0, 1.5, s) for s in enc.shapes])
    return enc


@pytest.mark.parametrize("arch,n_picks", [(oc.Arch(), 1000), (oc.Arch(arm_ctx=8, syn_hidden=8), 300)])
def test_gradients_central_differences(arch, n_picks):
    """Random coordinates, central differences with eps 1e-3, rel 1e-4 (noise phase)."""
    enc = _small_encoder(arch)
    u = enc.noise(0)
    _, _, _, grads = enc.loss_and_grads(u)
    sizes = [t.numel() for t in enc.tensors]
    rng = np.random.default_rng(14)
    picks = [(ti, int(rng.integers(0, sizes[ti])))
             for ti in rng.choice(len(sizes), n_picks, p=np.array(sizes) / sum(sizes))]

    def loss_at():
        with torch.no_grad():
            return float(oc.forward(enc.x, enc.y, enc.P, arch, enc.train.lam, u, False)[0])

    checked = 0
    for ti, j in picks:
        t = enc.tensors[ti]
        flat = t.detach().view(-1)
        g = float(grads[ti].view(-1)[j])
        old = float(flat[j])

        def fd(eps):
            flat[j] = old + eps
            lp = loss_at()
            flat[j] = old - eps
            lm = loss_at()
            flat[j] = old
            return (lp - lm) / (2 * eps)

        tol = 2.5e-5 * max(abs(g), 1e-4)
        f1, f2 = fd(1e-3), fd(5e-4)
        if abs(f1 - f2) <= tol:
            ref = f1
        else:  # a ReLU / clamp kink lies between eps/2 and eps: halve once more
            f3 = fd(2.5e-4)
            if abs(f2 - f3) > tol:
                continue
            ref = f2
        checked += 1
        assert abs(ref - g) <= 1e-4 * max(abs(g), 1e-4), (ti, j, g, ref)
    assert checked > 0.9 * n_picks


def test_ste_gradient_equals_noise_gradient_at_rounding_offset():
    """Hard phase: dL/dy is the gradient at y_hat = rint(y), i.e. the noise-phase gradient
    with u = rint(y) - y."""
    arch = oc.Arch(arm_ctx=8, syn_hidden=8)
    enc = _small_encoder(arch)
    _, _, _, g_hard = enc.loss_and_grads(hard=True)
    u = [torch.round(y.detach()) - y.detach() for y in enc.y]
    _, _, _, g_noise = enc.loss_and_grads(u_levels=u, hard=False)
    for a, b in zip(g_hard, g_noise):
        assert torch.max(torch.abs(a - b)) < 1e-12


def test_adam_first_step_is_lr_sign():
    arch = oc.Arch(arm_ctx=8, syn_hidden=8)
    enc = _small_encoder(arch)
    before = [t.detach().clone() for t in enc.tensors]
    _, _, _, grads = enc.loss_and_grads()
    enc.adam_update(grads)
    lr = enc.train.lr
    for b, a, g in zip(before, enc.tensors, grads):
        big = torch.abs(g) > 1e-4
        step = (a.detach() - b)[big]
        assert torch.max(torch.abs(step + lr * torch.sign(g[big]))) < lr * 1e-3


def test_training_reduces_rd_cost():
    arch = oc.Arch(arm_ctx=8, syn_hidden=8)
    enc = oc.OracleEncoder(syn.synthetic_image(32, 32, 0), arch, oc.Train(lam=1e-3, total_iters=40),
                           syn.initial_parameters(syn.ArchSizes(arm_ctx=8, syn_hidden=8), 0))
    first = enc.step()[0]
    for _ in range(39):
        last = enc.step()[0]
    assert last < 0.5 * first


# ---------------------------------------------------------------- C3 soft-rounding proxy

def test_soft_round_fixed_points_and_symmetry():
    """Integers and half-integers are fixed points; s_T(-x) = -s_T(x); strictly increasing."""
    for T in (0.05, 0.3, 1.0, 4.0):
        k = torch.arange(-6, 7, dtype=torch.float64)
        assert torch.max(torch.abs(oc.soft_round(k, T) - k)) < 1e-12
        assert torch.max(torch.abs(oc.soft_round(k + 0.5, T) - (k + 0.5))) < 1e-12
        x = torch.linspace(-4.9, 4.9, 2001, dtype=torch.float64)
        assert torch.max(torch.abs(oc.soft_round(-x, T) + oc.soft_round(x, T))) < 1e-12
        assert bool(torch.all(torch.diff(oc.soft_round(x, T)) > 0))


def test_soft_round_continuous_across_integers():
    for T in (0.1, 0.3, 2.0):
        for n in (-2.0, 0.0, 3.0):
            lo = oc.soft_round(torch.tensor(n - 1e-9, dtype=torch.float64), T)
            hi = oc.soft_round(torch.tensor(n + 1e-9, dtype=torch.float64), T)
            assert abs(float(hi - lo)) < 1e-6


def test_soft_round_limits():
    """T -> 0: rounding (away from the half-integers); large T: the identity."""
    x = torch.tensor([-2.3, -1.2, -0.1, 0.2, 0.7, 1.4, 2.95], dtype=torch.float64)
    assert torch.equal(oc.soft_round(x, 1e-3), torch.round(x))
    assert torch.max(torch.abs(oc.soft_round(x, 1e3) - x)) < 1e-6


def test_soft_proxy_gradient_central_differences():
    """d/dy of s_T(s_T(y) + u) by autograd matches central differences of the proxy."""
    rng = np.random.default_rng(5)
    for T in (0.1, 0.3, 1.0):
        y = torch.tensor(rng.normal(0, 2, 200), dtype=torch.float64, requires_grad=True)
        u = torch.tensor(rng.uniform(-0.5, 0.5, 200), dtype=torch.float64)
        (g,) = torch.autograd.grad(oc.quantize(y, u, False, T).sum(), y)
        eps = 1e-6
        with torch.no_grad():
            fd = (oc.quantize(y + eps, u, False, T) - oc.quantize(y - eps, u, False, T)) / (2 * eps)
        # relative error, with an absolute floor where the derivative is tiny (flat steps)
        assert torch.max(torch.abs(fd - g) / torch.clamp(torch.abs(g), min=1e-4)) < 1e-5


def test_soft_proxy_loss_gradients_central_differences():
    """The whole loss with the soft proxy: latent gradients against central differences."""
    arch = oc.Arch(arm_ctx=8, syn_hidden=8)
    enc = _small_encoder(arch)
    enc.train = oc.Train(lam=enc.train.lam, total_iters=100, soft_temp=0.3)
    u = enc.noise(0)
    _, _, _, grads = enc.loss_and_grads(u)
    rng = np.random.default_rng(21)
    checked = 0
    for _ in range(200):
        l = int(rng.integers(0, len(enc.y)))
        t = enc.y[l]
        flat = t.detach().view(-1)
        j = int(rng.integers(0, flat.numel()))
        g = float(grads[l].view(-1)[j])
        old = float(flat[j])

        def loss_at():
            with torch.no_grad():
                return float(oc.forward(enc.x, enc.y, enc.P, arch, enc.train.lam, u, False, 0.3)[0])

        def fd(eps):
            flat[j] = old + eps
            lp = loss_at()
            flat[j] = old - eps
            lm = loss_at()
            flat[j] = old
            return (lp - lm) / (2 * eps)

        tol = 2.5e-5 * max(abs(g), 1e-4)
        f1, f2 = fd(1e-4), fd(5e-5)
        if abs(f1 - f2) > tol:   # a kink between the two steps
            continue
        checked += 1
        assert abs(f1 - g) <= 1e-4 * max(abs(g), 1e-4), (l, j, g, f1)
    assert checked > 150
