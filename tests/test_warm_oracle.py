"""Pins of the warm-start predictor oracle (oracle/warm.py): the convolution definition
by explicit loops, the whole forward wiring restated with tap loops, output sizes, the
constant-output case, gradients by central differences; and its parameter order against
the binding's."""
import numpy as np
import pytest
import torch

from oracle import warm as ow
from paper_2403_11651_gb300 import coolchic as cc
from paper_2403_11651_gb300 import synthetic as syn


def _params(seed=0, scale=1.0):
    flat = syn.warm_initial_parameters(seed).astype(np.float64) * scale
    P, k = {}, 0
    for name, shape in ow.param_shapes():
        n = int(np.prod(shape))
        P[name] = torch.tensor(flat[k:k + n].reshape(shape), dtype=ow.DT, requires_grad=True)
        k += n
    return P


def test_parameter_order_matches_binding():
    assert [(n, tuple(s)) for n, s in ow.param_shapes()] == \
        [(n, tuple(s)) for n, s in cc.WARM_LAYOUT]
    assert sum(int(np.prod(s)) for _, s in ow.param_shapes()) == syn.warm_initial_parameters(0).size


def test_conv_definition_by_loops():
    """torch's conv2d (stride 2, zero padding 1) equals the written-out sum."""
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 7, 9))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    got = torch.nn.functional.conv2d(torch.tensor(x)[None], torch.tensor(w), torch.tensor(b),
                                     stride=2, padding=1)[0].numpy()
    Ho, Wo = 4, 5
    want = np.zeros((4, Ho, Wo))
    for co in range(4):
        for y in range(Ho):
            for xx in range(Wo):
                acc = b[co]
                for ci in range(3):
                    for ky in range(3):
                        for kx in range(3):
                            iy, ix = 2 * y + ky - 1, 2 * xx + kx - 1
                            if 0 <= iy < 7 and 0 <= ix < 9:
                                acc += w[co, ci, ky, kx] * x[ci, iy, ix]
                want[co, y, xx] = acc
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("H,W", [(16, 16), (37, 53), (64, 40)])
def test_output_sizes_are_the_latent_levels(H, W):
    lv = ow.forward(torch.zeros(3, H, W, dtype=ow.DT), _params())
    assert [tuple(t.shape) for t in lv] == \
        [(-(-H // (1 << l)), -(-W // (1 << l))) for l in range(5)]


def test_zero_weights_give_the_biases():
    P = _params()
    with torch.no_grad():
        for n, t in P.items():
            if n.endswith(".w"):
                t.zero_()
            else:
                t.fill_(0.25)
    lv = ow.forward(torch.rand(3, 32, 48, dtype=ow.DT), P)
    assert torch.allclose(lv[0], torch.full_like(lv[0], 0.25))
    for t in lv[1:]:             # ReLU(0.25) through zero 1x1 weights: the head bias
        assert torch.allclose(t, torch.full_like(t, 0.25))


def test_gradients_central_differences():
    torch.manual_seed(0)
    x = torch.rand(3, 24, 32, dtype=ow.DT)
    P = _params(2)
    tg = [torch.randn(-(-24 // (1 << l)), -(-32 // (1 << l)), dtype=ow.DT) for l in range(5)]
    L = ow.loss(x, P, tg)
    L.backward()
    rng = np.random.default_rng(3)
    eps = 1e-6
    for name in ("c1.w", "c3.w", "c4.b", "h2.w", "h0.w", "h4.b"):
        t = P[name]
        for _ in range(3):
            i = tuple(int(rng.integers(s)) for s in t.shape)
            with torch.no_grad():
                t[i] += eps
                lp = float(ow.loss(x, P, tg))
                t[i] -= 2 * eps
                lm = float(ow.loss(x, P, tg))
                t[i] += eps
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - float(t.grad[i])) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, float(t.grad[i]))


def _conv_loops(x, w, b, s):
    """out[co, y, x] = b[co] + sum w[co, ci, ky, kx] in[ci, s y + ky - 1, s x + kx - 1]
    (0 outside), written out over the taps; x [Ci, H, W], w [Co, Ci, 3, 3]."""
    Ci, H, W = x.shape
    Ho, Wo = -(-H // s), -(-W // s)
    pad = np.zeros((Ci, H + 2 + s, W + 2 + s))
    pad[:, 1:H + 1, 1:W + 1] = x
    out = np.zeros((w.shape[0], Ho, Wo)) + b[:, None, None]
    for ky in range(3):
        for kx in range(3):
            win = pad[:, ky:ky + s * Ho:s, kx:kx + s * Wo:s]        # in[ci, s y + ky - 1, ...]
            out += np.einsum("oc,chw->ohw", w[:, :, ky, kx], win)
    return out


@pytest.mark.parametrize("H,W", [(16, 16), (21, 35)])
def test_forward_wiring_by_loops(H, W):
    """The architecture as written: level 0 = 3x3 stride-1 convolution of the image;
    a_1 .. a_4 = ReLU(3x3 stride-2 convolution of the previous stage, the image first);
    level l = 1x1 head of a_l.  Restated with explicit tap loops, not torch's conv2d."""
    rng = np.random.default_rng(H * W)
    x = rng.uniform(0, 1, (3, H, W))
    P = _params(5)
    Pn = {k: v.detach().numpy() for k, v in P.items()}
    want = [_conv_loops(x, Pn["h0.w"], Pn["h0.b"], 1)[0]]
    a = x
    for i in (1, 2, 3, 4):
        a = np.maximum(_conv_loops(a, Pn[f"c{i}.w"], Pn[f"c{i}.b"], 2), 0.0)
        want.append(np.einsum("c,chw->hw", Pn[f"h{i}.w"][0, :, 0, 0], a) + Pn[f"h{i}.b"][0])
    got = ow.forward(torch.tensor(x, dtype=ow.DT), P)
    for l in range(5):
        np.testing.assert_allclose(got[l].detach().numpy(), want[l], rtol=1e-12, atol=1e-12)


# ---- the BF16 reading of the tensor-core layers (conv 2 .. 4)

def test_bf16_rounding_is_nearest_even():
    """to_bf16 keeps 8 significand bits, rounding to nearest with ties to even; an FP64
    value goes through FP32 first (the GPU rounds its FP32 activations)."""
    u = 2.0 ** -7                                   # BF16 spacing just above 1
    cases = [(1.0 + u / 2, 1.0),                    # tie, 1.0 is even
             (1.0 + 3 * u / 2, 1.0 + 2 * u),        # tie, 1 + 2u is even
             (1.0 + u / 2 + 2.0 ** -20, 1.0 + u),   # above the tie
             (1.0 + u / 2 - 2.0 ** -20, 1.0),       # below the tie
             (-(1.0 + 3 * u / 2), -(1.0 + 2 * u)),
             (1.0 + u / 2 + 2.0 ** -40, 1.0),       # within FP32 rounding of the tie
             (0.75, 0.75), (0.0, 0.0)]
    got = ow.to_bf16(torch.tensor([c for c, _ in cases], dtype=torch.float64)).tolist()
    assert got == [e for _, e in cases]


def _bf16_rand(shape, gen):
    return ow.to_bf16(torch.randn(shape, generator=gen, dtype=torch.float64))


def test_bf16_conv_is_the_plain_conv_on_bf16_values():
    """With input, weights and output gradient already BF16 values the rounding does
    nothing: ConvBF16 equals the plain stride-2 convolution and its gradients."""
    gen = torch.Generator().manual_seed(3)
    a = _bf16_rand((1, 32, 11, 14), gen).requires_grad_(True)
    w = _bf16_rand((32, 32, 3, 3), gen).requires_grad_(True)
    b = torch.randn(32, generator=gen, dtype=torch.float64).requires_grad_(True)
    g = _bf16_rand((1, 32, 6, 7), gen)
    out = ow.ConvBF16.apply(a, w, b)
    da, dw, db = torch.autograd.grad(out, (a, w, b), g)
    ref = torch.nn.functional.conv2d(a, w, b, stride=2, padding=1)
    ra, rw, rb = torch.autograd.grad(ref, (a, w, b), g)
    assert torch.allclose(out, ref, rtol=1e-13, atol=1e-13)
    for x, y in ((da, ra), (dw, rw), (db, rb)):
        assert torch.allclose(x, y, rtol=1e-12, atol=1e-12)


def test_bf16_conv_rounds_every_operand():
    """On general values the forward moves by no more than the operands' rounding allows
    (relative 2^-9 each, so 2^-8 + 2^-18 per product), and does move; the backward uses the
    rounded output gradient: it equals the plain gradients of the rounded operands taken
    with the rounded output gradient, and differs from those with the unrounded one."""
    gen = torch.Generator().manual_seed(4)
    a = torch.randn((1, 32, 9, 10), generator=gen, dtype=torch.float64)
    w = torch.randn((32, 32, 3, 3), generator=gen, dtype=torch.float64)
    b = torch.randn(32, generator=gen, dtype=torch.float64)
    out = ow.ConvBF16.apply(a, w, b)
    plain = torch.nn.functional.conv2d(a, w, b, stride=2, padding=1)
    bound = torch.nn.functional.conv2d(a.abs(), w.abs(), None, stride=2, padding=1) * (2.0 ** -8 + 2.0 ** -18)
    assert bool(((out - plain).abs() <= bound).all())
    assert float((out - plain).abs().max()) > 0.0
    g = torch.randn(out.shape, generator=gen, dtype=torch.float64)
    ar = ow.to_bf16(a).requires_grad_(True)
    wr = ow.to_bf16(w).requires_grad_(True)
    br = b.clone().requires_grad_(True)
    a1, w1, b1 = a.clone().requires_grad_(True), w.clone().requires_grad_(True), b.clone().requires_grad_(True)
    got = torch.autograd.grad(ow.ConvBF16.apply(a1, w1, b1), (a1, w1, b1), g)
    ref = torch.autograd.grad(torch.nn.functional.conv2d(ar, wr, br, stride=2, padding=1),
                              (ar, wr, br), ow.to_bf16(g))
    unr = torch.autograd.grad(torch.nn.functional.conv2d(ar, wr, br, stride=2, padding=1),
                              (ar, wr, br), g)
    for x, y, z in zip(got, ref, unr):
        assert torch.allclose(x, y, rtol=1e-12, atol=1e-12)
        assert float((x - z).abs().max()) > 0.0


def test_bf16_predictor_close_to_fp64():
    """The BF16 reading changes the whole predictor's output by about BF16 precision."""
    x = torch.tensor(syn.synthetic_image(40, 56, 2).astype(np.float64) / 255.0).permute(2, 0, 1)
    P = _params(2)
    ref = ow.forward(x, P)
    got = ow.forward(x, P, bf16=True)
    assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])   # FP64 layers
    for l in (2, 3, 4):
        d = float((got[l] - ref[l]).abs().max())
        scale = float(ref[l].abs().max())
        assert 0.0 < d < 2e-2 * scale, (l, d, scale)


def test_step_work_count_matches_the_oracle_layers():
    """warm_bench's multiply-add count of a training step equals the one read off the
    oracle's layers: every convolution's output elements times its inputs per output, once
    forward, once for the weight gradient and once for the input gradient where one is
    needed (not into the image)."""
    from paper_2403_11651_gb300 import warm_bench
    for S in (64, 100, 512):
        x = torch.zeros(3, S, S, dtype=torch.float64)
        P = _params(0)
        a = x.unsqueeze(0)
        total = 0
        # head 0: forward and weight gradient
        total += 2 * S * S * 27
        for i in (1, 2, 3, 4):
            w = P[f"c{i}.w"]
            a = torch.relu(torch.nn.functional.conv2d(a, w, P[f"c{i}.b"], stride=2, padding=1))
            per_out = w.shape[1] * 9
            passes = 2 if i == 1 else 3
            total += passes * a.numel() * per_out
            total += 3 * a.shape[2] * a.shape[3] * w.shape[0]    # head i: forward, weight, input
        assert warm_bench.warm_macs_per_step(S) == total, S
