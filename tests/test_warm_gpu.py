"""Warm-start predictor on the GPU against the oracle (oracle/warm.py) in its BF16 reading
(conv 2 .. 4 on BF16 operands, every sum FP64): forward, loss and every parameter
gradient; Adam steps lower the loss.

Tolerances: the GPU accumulates in FP32 (relative 1e-6 over 288 terms), and where its FP32
value of an operand and the oracle's FP64 value fall on two sides of a BF16 rounding
boundary (a few elements per layer at these sizes) one operand differs by one BF16 unit
(2^-8 relative).  Predictions within 1e-3 of the largest value, the loss within
relative 1e-4, every parameter-gradient group within 2e-3 of its largest entry.  The
prediction of levels 2 .. 4 must also be at least three times closer to the BF16 reading
than to the FP64 one: the tensor-core layers really take BF16 operands."""
import numpy as np
import pytest
import torch

from oracle import warm as ow
from paper_2403_11651_gb300 import coolchic as cc
from paper_2403_11651_gb300 import synthetic as syn

from .helpers import assert_group_close

pytestmark = pytest.mark.gpu


def _oracle(flat):
    P, k = {}, 0
    for name, shape in ow.param_shapes():
        n = int(np.prod(shape))
        P[name] = torch.tensor(flat[k:k + n].astype(np.float64).reshape(shape),
                               requires_grad=True)
        k += n
    return P


@pytest.mark.parametrize("H,W,seed", [(64, 96, 0), (37, 53, 1), (256, 256, 2)])
def test_forward_loss_gradients(H, W, seed):
    flat = syn.warm_initial_parameters(seed)
    rgb = syn.synthetic_image(H, W, seed)
    shapes = [(-(-H // (1 << l)), -(-W // (1 << l))) for l in range(7)]
    rng = np.random.default_rng(seed)
    target = [rng.normal(0, 1.0, s).astype(np.float32) for s in shapes]
    flat_t = np.concatenate([t.ravel() for t in target])
    n_lat = flat_t.size
    w = cc.cc_warm_create(H, W, flat)
    try:
        pred = cc.cc_warm_predict(w, rgb, n_lat)
        g = np.empty(flat.size, np.float32)
        loss = cc.cc_warm_loss_grad(w, rgb, flat_t, g)
    finally:
        cc.cc_warm_free(w)
    x = torch.tensor(rgb.astype(np.float64) / 255.0).permute(2, 0, 1).contiguous()
    P = _oracle(flat)
    ref = ow.forward(x, P, bf16=True)
    ref64 = ow.forward(x, P)
    k = 0
    for l, (h, ww) in enumerate(shapes):
        got = pred[k:k + h * ww].reshape(h, ww)
        if l < 5:
            r = ref[l].detach().numpy()
            err = np.abs(got - r).max()
            assert err <= 1e-3 * max(1.0, float(np.abs(r).max())), (l, err)
            if l >= 2:
                err64 = np.abs(got - ref64[l].detach().numpy()).max()
                assert 3 * err <= err64, (l, err, err64)
        else:
            assert not got.any()
        k += h * ww
    L = ow.loss(x, P, [torch.tensor(t.astype(np.float64)) for t in target[:5]], bf16=True)
    L.backward()
    assert abs(loss - float(L)) <= 1e-4 * float(L)
    k = 0
    for name, shape in ow.param_shapes():
        n = int(np.prod(shape))
        assert_group_close(g[k:k + n].reshape(shape), P[name].grad.numpy(), 2e-3, name)
        k += n


def test_training_lowers_the_loss():
    H, W = 64, 64
    rgb = syn.synthetic_image(H, W, 5)
    shapes = [(-(-H // (1 << l)), -(-W // (1 << l))) for l in range(7)]
    x = rgb.astype(np.float32).mean(axis=2) / 255.0
    # a target the predictor can reach: the image's mean intensity, pooled per level
    target = []
    for l, (h, w) in enumerate(shapes):
        f = 1 << l
        pad = np.pad(x, ((0, h * f - H), (0, w * f - W)), mode="edge")
        target.append((pad.reshape(h, f, w, f).mean(axis=(1, 3)) * 4.0 - 2.0).astype(np.float32))
    flat_t = np.concatenate([t.ravel() for t in target])
    w = cc.cc_warm_create(H, W, syn.warm_initial_parameters(5))
    try:
        first = cc.cc_warm_train_step(w, rgb, flat_t, 1e-3)
        for _ in range(200):
            last = cc.cc_warm_train_step(w, rgb, flat_t, 1e-3)
    finally:
        cc.cc_warm_free(w)
    assert last < 0.4 * first, (first, last)


def test_host_and_device_buffers_agree():
    """Image, target and outputs may each be host or device memory: same results."""
    H, W = 48, 80
    flat = syn.warm_initial_parameters(3)
    rgb = syn.synthetic_image(H, W, 3)
    n_lat = sum(-(-H // (1 << l)) * -(-W // (1 << l)) for l in range(7))
    tgt = np.random.default_rng(3).normal(0, 1.0, n_lat).astype(np.float32)
    d_flat, d_rgb, d_tgt = (torch.from_numpy(a).cuda() for a in (flat, rgb, tgt))
    g_dev = torch.empty(flat.size, dtype=torch.float32, device="cuda")
    p_dev = torch.empty(n_lat, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    w = cc.cc_warm_create(H, W, d_flat)
    try:
        g_host = np.empty(flat.size, np.float32)
        l_host = cc.cc_warm_loss_grad(w, rgb, tgt, g_host)
        l_dev = cc.cc_warm_loss_grad(w, d_rgb, d_tgt, g_dev)
        p_host = cc.cc_warm_predict(w, rgb, n_lat)
        cc.cc_warm_predict(w, d_rgb, n_lat, p_dev)
    finally:
        cc.cc_warm_free(w)
    assert l_host == l_dev
    assert np.array_equal(g_host, g_dev.cpu().numpy())
    assert np.array_equal(p_host, p_dev.cpu().numpy())


def test_train_step_loss_destinations_agree():
    """A training step replays captured graphs; the loss can go to host memory (checked,
    synchronising), to device memory (queued) or nowhere.  All three give the same
    parameters bit for bit, and the same losses."""
    H, W = 40, 72
    flat = syn.warm_initial_parameters(7)
    rgb = torch.from_numpy(syn.synthetic_image(H, W, 7)).cuda()
    n_lat = sum(-(-H // (1 << l)) * -(-W // (1 << l)) for l in range(7))
    tgt = torch.from_numpy(np.random.default_rng(7).normal(0, 1.0, n_lat).astype(np.float32)).cuda()
    d_loss = torch.zeros(6, dtype=torch.float64, device="cuda")
    out, host = [], []
    for mode in ("host", "device", "none"):
        w = cc.cc_warm_create(H, W, flat)
        try:
            for k in range(6):
                lr = 1e-3 if k < 3 else 5e-4
                if mode == "host":
                    host.append(cc.cc_warm_train_step(w, rgb, tgt, lr))
                elif mode == "device":
                    cc.cc_warm_train_step(w, rgb, tgt, lr, loss_out=d_loss[k])
                else:
                    cc.cc_warm_train_step(w, rgb, tgt, lr, with_loss=False)
            out.append(cc.cc_warm_get_params(w))
        finally:
            cc.cc_warm_free(w)
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
    assert host == d_loss.cpu().tolist()
    assert not np.array_equal(out[0], flat)
