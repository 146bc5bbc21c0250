"""Parity of the CUDA path (through its C ABI) with the FP64 oracle, on a GB300.

Tolerances (stated for this workload): forward rate and distortion rel 1e-5; gradients
rel 1e-4 of each tensor's largest magnitude (per latent level and per parameter tensor);
the first 10 training iterations' losses rel 1e-4; final RD cost within 1 %; the
quantisation noise bit-exact.
"""
import ctypes
import json
import os

import numpy as np
import pytest
import torch

from oracle import coolchic as oc
from oracle import philox
from paper_2403_11651_gb300 import coolchic as cc
from paper_2403_11651_gb300 import synthetic as syn

from .helpers import (Pair, assert_group_close, assert_latents_close_with_ties, config_dict,
                      margins)

pytestmark = pytest.mark.gpu

SIZES = [(64, 48), (67, 45), (16, 24)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    cc.load()


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("H,W", [(67, 45), (512, 768), (1, 1)])
def test_noise_bit_exact(H, W):
    p = Pair(config_dict("c2"), H, W, seed=12345678901)
    try:
        for it in (0, 7, 123456):
            got = cc.cc_noise(p.ctx, it, p.n_lat)
            ref = np.concatenate([u.ravel() for u in
                                  philox.latent_noise(12345678901, it, oc.level_shapes(H, W))])
            assert np.array_equal(got.astype(np.float64), ref)
    finally:
        p.close()


@pytest.mark.parametrize("arch", ["c1", "c2", "t300", "t545", "t1079"])
@pytest.mark.parametrize("H,W", SIZES)
def test_forward_and_gradients(arch, H, W):
    p = Pair(config_dict(arch, lam=1e-2), H, W, seed=3, random_state=True)
    try:
        u = syn.uniform_noise(H, W, 5)
        gy, gp, D, R = p.gpu_grads(u, hard=0)
        ry, rp, rD, rR = p.oracle_grads(u)
        assert _rel(D, rD) < 1e-5, (D, rD)
        assert _rel(R, rR) < 1e-5, (R, rR)
        for l in range(7):
            assert_group_close(gy[l], ry[l], 1e-4, f"dL/dy level {l}")
        for k in rp:
            assert_group_close(gp[k], rp[k], 1e-4, k)
    finally:
        p.close()


@pytest.mark.parametrize("arch", ["c1", "c2"])
def test_hard_rounding_pass(arch):
    H, W = 40, 56
    p = Pair(config_dict(arch, lam=1e-2), H, W, seed=4, random_state=True)
    try:
        gy, gp, D, R = p.gpu_grads(None, hard=1)
        ry, rp, rD, rR = p.oracle_grads(None, hard=True)
        assert _rel(D, rD) < 1e-5 and _rel(R, rR) < 1e-5
        for l in range(7):
            assert_group_close(gy[l], ry[l], 1e-4, f"level {l}")
        for k in rp:
            assert_group_close(gp[k], rp[k], 1e-4, k)
        Dg, Rg, Cg = cc.cc_rd_cost(p.ctx, True)
        Do, Ro, Co = p.oracle.rd_cost(hard=True)
        assert _rel(Dg, Do) < 1e-5 and _rel(Rg, Ro) < 1e-5 and _rel(Cg, Co) < 1e-5
    finally:
        p.close()


def test_decode_matches_oracle():
    H, W = 48, 80
    p = Pair(config_dict("c2"), H, W, seed=6, random_state=True)
    try:
        got = cc.cc_decode(p.ctx, H, W)
        ref = p.oracle.decode()
        assert np.max(np.abs(got - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))
    finally:
        p.close()


# seeds whose oracle state has no decision (ReLU pre-activation, rate floor, scale clamp)
# within 1e-6 of its tie, where FP32 and FP64 may both be right and differ
@pytest.mark.parametrize("arch,H,W,seed", [("c1", 67, 45, 9), ("c1", 130, 97, 9),
                                           ("c2", 67, 45, 9), ("c2", 130, 97, 11),
                                           ("t1079", 67, 45, 9), ("t1079", 130, 97, 10)])
def test_soft_rounding_forward_and_gradients(arch, H, W, seed):
    """C3 soft-rounding proxy (temperature 0.3): D, R and every gradient against the oracle."""
    p = Pair(config_dict(arch, lam=1e-2, soft_temp=0.3), H, W, seed=seed, random_state=True)
    try:
        u = syn.uniform_noise(H, W, 6)
        gy, gp, D, R = p.gpu_grads(u, hard=0)
        ry, rp, rD, rR = p.oracle_grads(u)
        assert _rel(D, rD) < 1e-5, (D, rD)
        assert _rel(R, rR) < 1e-5, (R, rR)
        arm_m, syn_m = margins(p, u)
        offs = oc.causal_offsets(p.d["arm_ctx"])
        for l in range(7):
            assert_latents_close_with_ties(gy[l], ry[l], l, arm_m[l], syn_m, offs, 1e-4,
                                           max_outliers=len(offs) + 1)
        for k in rp:
            assert_group_close(gp[k], rp[k], 1e-4, k)
    finally:
        p.close()


def test_soft_rounding_iterations():
    """Ten iterations on the soft proxy's noise phase, then ten straight-through ones."""
    p = Pair(config_dict("c1", total_iters=20, ste_frac=0.5, soft_temp=0.3), 64, 64, seed=8)
    try:
        cc.cc_encode_iters(p.ctx, 20)
        got = cc.cc_get_losses(p.ctx, 0, 20)
        for t in range(20):
            loss, D, R = p.oracle.step()
            tol = 1e-4 if t < 10 else 1e-3
            assert _rel(got[t, 2], loss) < tol, (t, got[t], loss)
    finally:
        p.close()


@pytest.mark.parametrize("arch,H,W", [("c1", 64, 64), ("c2", 64, 96), ("c2", 67, 45)])
def test_first_ten_iterations(arch, H, W):
    p = Pair(config_dict(arch, total_iters=20, ste_frac=0.5), H, W, seed=7)
    try:
        cc.cc_encode_iters(p.ctx, 10)
        got = cc.cc_get_losses(p.ctx, 0, 10)
        for t in range(10):
            loss, D, R = p.oracle.step()
            assert _rel(got[t, 0], D) < 1e-4, (t, got[t], D)
            assert _rel(got[t, 1], R) < 1e-4, (t, got[t], R)
            assert _rel(got[t, 2], loss) < 1e-4, (t, got[t], loss)
        # iterations 10..19 use straight-through rounding (ste_frac 0.5)
        cc.cc_encode_iters(p.ctx, 10)
        got = cc.cc_get_losses(p.ctx, 10, 10)
        for t in range(10):
            loss, D, R = p.oracle.step()
            assert _rel(got[t, 2], loss) < 1e-3, (t, got[t], loss)
    finally:
        p.close()


def test_c2_full_size_iterations():
    """512x768 with the 2300-MAC decoder through cc_encode_iters, in the launch
    configuration the bench times: one replay of the 16-iteration graph (the ARM kernel on
    its side stream beside the upsampling / synthesis chain, programmatic dependent
    launches, the latent and parameter updates finishing the pass from two streams), then
    four replays of the one-iteration graph.  A 20-iteration schedule whose last half is
    straight-through: the first 10 iterations' D, R and loss at rel 1e-4, the next 10 at
    rel 1e-3 (Sec. II eq. (1) per iteration; Adam as in Sec. IV-B)."""
    d = config_dict("c2", total_iters=20, ste_frac=0.5)
    H, W = 512, 768
    p = Pair(d, H, W, seed=0)
    try:
        cc.cc_encode_iters(p.ctx, 16)
        cc.cc_encode_iters(p.ctx, 4)
        got = cc.cc_get_losses(p.ctx, 0, 20)
        for t in range(20):
            loss, D, R = p.oracle.step()
            tol = 1e-4 if t < 10 else 1e-3
            assert _rel(got[t, 0], D) < tol, (t, got[t], D)
            assert _rel(got[t, 1], R) < tol, (t, got[t], R)
            assert _rel(got[t, 2], loss) < tol, (t, got[t], loss)
        Dg, Rg, Cg = cc.cc_rd_cost(p.ctx, True)
        Do, Ro, Co = p.oracle.rd_cost(hard=True)
        assert _rel(Cg, Co) < 1e-3, ((Dg, Rg, Cg), (Do, Ro, Co))
    finally:
        p.close()


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_c1_final_rd_cost(seed):
    """256x256, 50 Adam iterations (the first configuration): final RD cost within 1 %."""
    d = cc.load_config("c1")
    p = Pair(d, d["H"], d["W"], seed=seed)
    try:
        cc.cc_encode_iters(p.ctx, d["total_iters"])
        for _ in range(d["total_iters"]):
            p.oracle.step()
        g = cc.cc_rd_cost(p.ctx, True)
        o = p.oracle.rd_cost(hard=True)
        assert _rel(g[2], o[2]) < 1e-2, (g, o)
    finally:
        p.close()


def test_c2_full_size_gradients():
    """512x768 with the 2300-MAC decoder, in the launch configuration the bench times.

    Over 524 256 latents a handful of ReLU / floor decisions sit within FP32 rounding of
    their tie; there the two one-sided derivatives are both correct.  Latents whose
    gradient depends on such a decision (found by the oracle) are exempt, every other
    element must agree to rel 1e-4.
    """
    d = cc.load_config("c2")
    p = Pair(d, d["H"], d["W"], seed=0, random_state=True, state_scale=2.0)
    try:
        u = syn.uniform_noise(d["H"], d["W"], 9)
        gy, gp, D, R = p.gpu_grads(u, hard=0)
        ry, rp, rD, rR = p.oracle_grads(u)
        assert _rel(D, rD) < 1e-5 and _rel(R, rR) < 1e-5
        arm_m, syn_m = margins(p, u)
        offs = oc.causal_offsets(d["arm_ctx"])
        for l in range(7):
            assert_latents_close_with_ties(gy[l], ry[l], l, arm_m[l], syn_m, offs, 1e-4)
        for k in rp:
            assert_group_close(gp[k], rp[k], 1e-4, k)
    finally:
        p.close()


def test_c2_final_rd_cost_golden(golden_dir):
    """10 000 iterations (last 20 % straight-through) against the stored oracle run.

    FP32 and FP64 runs of 10^4 Adam steps decorrelate (the loss moves by ~3 % between
    samples 100 iterations apart in the stored run); what must agree is where they end up.
    Tolerances from measured spreads: the GPU's final hard cost over six noise seeds from
    the same initial state has a standard deviation of 1.6 % of its mean, so the final
    hard cost must lie within 3 of those (5 %); the mean training loss over the oracle's
    21 stored samples from iteration 8000 on (per-sample spread 3.1 %, so ~0.7 % on a
    mean) must agree within 2 %."""
    path = os.path.join(golden_dir, "c2_lam1e-3.json")
    if not os.path.exists(path):
        pytest.skip("stored oracle run not present")
    with open(path) as f:
        ref = json.load(f)
    d = cc.load_config("c2")
    cfg = cc.make_config(d, seed=ref["seed"], lam=ref["lam"])
    rgb = syn.synthetic_image(d["H"], d["W"], ref["seed"])
    init = cc.flatten_params(syn.initial_parameters(syn.ArchSizes.from_config(d), ref["seed"]), cfg)
    ctx = cc.cc_init_image(cfg, rgb, d["H"], d["W"], init)
    try:
        cc.cc_encode_iters(ctx, ref["iters"])
        D, R, cost = cc.cc_rd_cost(ctx, True)
        first = ref["iters"] - 2000
        log = cc.cc_get_losses(ctx, first, 2000)           # rows: D, R, loss
    finally:
        cc.cc_free(ctx)
    traj = np.array(ref["trajectory"])
    late = traj[traj[:, 0] >= first]
    gpu_mean = log[late[:, 0].astype(int) - first, 2].mean()
    assert _rel(gpu_mean, late[:, 1].mean()) < 0.02, (gpu_mean, late[:, 1].mean())
    assert _rel(cost, ref["final_hard"]["cost"]) < 0.05, (cost, ref["final_hard"])


def test_deterministic_and_resume():
    d = config_dict("c2", total_iters=40, ste_frac=0.25)
    a = Pair(d, 48, 64, seed=8)
    b = Pair(d, 48, 64, seed=8)
    try:
        cc.cc_encode_iters(a.ctx, 20)
        blob = cc.cc_get_state(a.ctx)
        cc.cc_encode_iters(a.ctx, 20)
        la = cc.cc_get_losses(a.ctx, 20, 20)
        cc.cc_set_state(b.ctx, blob)
        assert cc.cc_iteration(b.ctx) == 20
        cc.cc_encode_iters(b.ctx, 20)
        lb = cc.cc_get_losses(b.ctx, 20, 20)
        assert np.array_equal(la, lb)
        assert cc.cc_get_state(a.ctx) == cc.cc_get_state(b.ctx)
    finally:
        a.close()
        b.close()


def test_workspace_from_torch_matches():
    d = config_dict("c1")
    H, W = 40, 40
    cfg = cc.make_config(d, seed=2)
    rgb = syn.synthetic_image(H, W, 2)
    init = cc.flatten_params(syn.initial_parameters(syn.ArchSizes.from_config(d), 2), cfg)
    n = cc.cc_workspace_size(cfg, H, W)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    c1 = cc.cc_init_image_ws(cfg, torch.from_numpy(rgb).cuda(), H, W, torch.from_numpy(init).cuda(),
                             st, ws, n)
    c2 = cc.cc_init_image(cfg, rgb, H, W, init)
    try:
        # contexts of one device share its weight banks: run them one after the other
        cc.cc_encode_iters(c1, 12)
        st.synchronize()
        cc.cc_encode_iters(c2, 12)
        torch.cuda.synchronize()
        assert np.array_equal(cc.cc_get_losses(c1, 0, 12), cc.cc_get_losses(c2, 0, 12))
        with pytest.raises(cc.CCError):
            cc.cc_init_image_ws(cfg, rgb, H, W, init, None, ws, n - 1)
    finally:
        cc.cc_free(c1)
        cc.cc_free(c2)


def test_bad_state_blob_rejected():
    p = Pair(config_dict("c1"), 16, 16, seed=1)
    q = Pair(config_dict("c1"), 16, 24, seed=1)
    try:
        blob = cc.cc_get_state(p.ctx)
        with pytest.raises(cc.CCError) as e:
            cc.cc_set_state(q.ctx, blob)
        assert e.value.code == cc.CC_ESTATE
        with pytest.raises(cc.CCError):
            cc.cc_set_state(p.ctx, blob[:-4])
    finally:
        p.close()
        q.close()


def test_losses_async_matches_sync():
    """cc_get_losses_async copies the same log entries as cc_get_losses, across the ring's
    wrap-around, into pinned host or device memory; evicted entries are refused."""
    d = config_dict("c1", total_iters=5000)
    H, W = 32, 32
    cfg = cc.make_config(d, seed=4)
    rgb = syn.synthetic_image(H, W, 4)
    ctx = cc.cc_init_image(cfg, rgb, H, W)
    try:
        cc.cc_encode_iters(ctx, 4100)
        ref = cc.cc_get_losses(ctx, 4, 4096)
        host = torch.zeros((4096, 3), dtype=torch.float64).pin_memory()
        cc.cc_get_losses_async(ctx, 4, 4096, host)
        dev = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
        cc.cc_get_losses_async(ctx, 4090, 10, dev)
        torch.cuda.synchronize()
        assert np.array_equal(host.numpy(), ref)
        assert np.array_equal(dev.cpu().numpy(), ref[-10:])
        with pytest.raises(cc.CCError):
            cc.cc_get_losses_async(ctx, 3, 1, host)
        with pytest.raises(cc.CCError):
            cc.cc_get_losses_async(ctx, 4099, 2, host)
    finally:
        cc.cc_free(ctx)


def test_set_image_replaces_the_image():
    """After cc_set_image (pinned host or device source) a context iterates exactly as a
    context created with that image."""
    d = config_dict("c1")
    H, W = 40, 56
    cfg = cc.make_config(d, seed=5)
    img_a, img_b = syn.synthetic_image(H, W, 5), syn.synthetic_image(H, W, 6)
    init = cc.flatten_params(syn.initial_parameters(syn.ArchSizes.from_config(d), 5), cfg)
    ca = cc.cc_init_image(cfg, img_a, H, W, init)
    cb = cc.cc_init_image(cfg, img_b, H, W, init)
    cc2 = cc.cc_init_image(cfg, img_b, H, W, init)
    try:
        cc.cc_set_image(ca, torch.from_numpy(img_b).pin_memory())
        cc.cc_encode_iters(ca, 5)
        la = cc.cc_get_losses(ca, 0, 5)
        cc.cc_encode_iters(cb, 5)
        lb = cc.cc_get_losses(cb, 0, 5)
        assert np.array_equal(la, lb)
        cc.cc_set_image(cc2, torch.from_numpy(img_a).cuda())
        cc.cc_set_image(cc2, torch.from_numpy(img_b).cuda())
        cc.cc_encode_iters(cc2, 5)
        assert np.array_equal(cc.cc_get_losses(cc2, 0, 5), lb)
    finally:
        for c in (ca, cb, cc2):
            cc.cc_free(c)


def test_autograd_function_matches_oracle():
    """CoolChicIter: the loss of eq. (1) and, through loss.backward(), the hand-written
    gradients -- against the FP64 oracle; a few torch.optim.Adam steps through it lower
    the loss."""
    from paper_2403_11651_gb300.autograd import coolchic_loss
    H, W = 40, 56
    p = Pair(config_dict("c1", lam=1e-2), H, W, seed=3, random_state=True)
    try:
        u = syn.uniform_noise(H, W, 5)
        noise = torch.from_numpy(np.concatenate([a.ravel() for a in u])).cuda()
        y = torch.from_numpy(cc.cc_get_latents(p.ctx, p.n_lat)).cuda().requires_grad_()
        prm = torch.from_numpy(cc.cc_get_params(p.ctx, p.n_params)).cuda().requires_grad_()
        loss = coolchic_loss(p.ctx, y, prm, noise, hard=0)
        loss.backward()
        ry, rp, rD, rR = p.oracle_grads(u)
        assert _rel(float(loss.detach()), rD + 1e-2 * rR) < 1e-5
        gy = cc.split_latents(y.grad.cpu().numpy(), H, W)
        for l in range(7):
            assert_group_close(gy[l], ry[l], 1e-4, f"dL/dy level {l}")
        gp = cc.unflatten_params(prm.grad.cpu().numpy(), p.cfg)
        for k in rp:
            assert_group_close(gp[k], rp[k], 1e-4, k)
        # optimisation through the Function (PyTorch's Adam)
        opt = torch.optim.Adam([y, prm], lr=1e-2)
        first = None
        for _ in range(30):
            opt.zero_grad()
            l = coolchic_loss(p.ctx, y, prm, noise, hard=0)
            l.backward()
            opt.step()
            first = float(l.detach()) if first is None else first
        assert float(coolchic_loss(p.ctx, y, prm, noise, hard=0).detach()) < 0.9 * first
    finally:
        p.close()


def test_nan_latent_reported():
    """A NaN written into the latents through the C ABI (a host-side fault) makes the next
    cost evaluation report CC_ENONFINITE instead of a number."""
    p = Pair(config_dict("c1"), 32, 48, seed=2)
    try:
        y = cc.cc_get_latents(p.ctx, p.n_lat)
        y[5] = np.nan
        cc.cc_set_latents(p.ctx, y)
        D, R, C = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        code = cc._lib().cc_rd_cost(p.ctx, 1, ctypes.byref(D), ctypes.byref(R), ctypes.byref(C))
        assert code == cc.CC_ENONFINITE
        y[5] = 0.0                      # writing finite latents clears the condition
        cc.cc_set_latents(p.ctx, y)
        assert cc._lib().cc_rd_cost(p.ctx, 1, ctypes.byref(D), ctypes.byref(R),
                                    ctypes.byref(C)) == cc.CC_OK
    finally:
        p.close()


def test_nonfinite_chunk_rolls_back():
    """A NaN gradient injected at iteration 27 (host-side request, one shot) poisons the
    chunk of iterations 20..29: cc_encode_iters_checked restores the state from before the
    chunk and reports CC_ENONFINITE; continuing from there reproduces an undisturbed run
    bit for bit."""
    d = config_dict("c1", total_iters=100)
    a = Pair(d, 48, 64, seed=3)
    b = Pair(d, 48, 64, seed=3)
    try:
        assert cc.cc_encode_iters_checked(a.ctx, 20, 10) == (cc.CC_OK, 20)
        cc.cc_encode_iters(b.ctx, 20)
        before = cc.cc_get_state(a.ctx)
        cc.cc_debug_inject(a.ctx, cc.CC_FAULT_NAN_GRAD, 27)
        code, done = cc.cc_encode_iters_checked(a.ctx, 30, 10)
        assert (code, done) == (cc.CC_ENONFINITE, 0)
        assert cc.cc_iteration(a.ctx) == 20
        assert cc.cc_get_state(a.ctx) == before
        assert cc.cc_encode_iters_checked(a.ctx, 30, 10) == (cc.CC_OK, 30)
        cc.cc_encode_iters(b.ctx, 30)
        assert np.array_equal(cc.cc_get_losses(a.ctx, 20, 30), cc.cc_get_losses(b.ctx, 20, 30))
        assert cc.cc_get_state(a.ctx) == cc.cc_get_state(b.ctx)
    finally:
        a.close()
        b.close()


def test_injected_allocation_failure():
    """CC_FAULT_ALLOC: the next context creation fails with CC_ENOMEM (nothing allocated,
    nothing leaked); the one after succeeds."""
    d = config_dict("c1")
    cfg = cc.make_config(d, seed=1)
    rgb = syn.synthetic_image(16, 16, 1)
    cc.cc_debug_inject(None, cc.CC_FAULT_ALLOC)
    with pytest.raises(cc.CCError) as e:
        cc.cc_init_image(cfg, rgb, 16, 16)
    assert e.value.code == cc.CC_ENOMEM
    ctx = cc.cc_init_image(cfg, rgb, 16, 16)
    cc.cc_free(ctx)


def test_arm_wait_timeout_rolls_back():
    """A wait that nothing completes: asked from the host, every CTA of the ARM kernel
    leaves out its first context load, its bounded wait runs out, it records the fault,
    waits for its loads in flight and returns.  cc_encode_iters_checked reports
    CC_ETIMEOUT and restores the state from before the chunk; the context then runs on
    bit-identical to an undisturbed one."""
    d = config_dict("c2", total_iters=100)
    a = Pair(d, 48, 64, seed=4)
    b = Pair(d, 48, 64, seed=4)
    try:
        assert cc.cc_encode_iters_checked(a.ctx, 20, 10) == (cc.CC_OK, 20)
        cc.cc_encode_iters(b.ctx, 20)
        before = cc.cc_get_state(a.ctx)
        cc.cc_debug_inject(a.ctx, cc.CC_FAULT_ARM_STALL)
        code, done = cc.cc_encode_iters_checked(a.ctx, 30, 10)
        assert (code, done) == (cc.CC_ETIMEOUT, 0)
        assert cc.cc_iteration(a.ctx) == 20
        assert cc.cc_get_state(a.ctx) == before
        assert cc.cc_encode_iters_checked(a.ctx, 30, 10) == (cc.CC_OK, 30)
        cc.cc_encode_iters(b.ctx, 30)
        assert np.array_equal(cc.cc_get_losses(a.ctx, 20, 30), cc.cc_get_losses(b.ctx, 20, 30))
        assert cc.cc_get_state(a.ctx) == cc.cc_get_state(b.ctx)
    finally:
        a.close()
        b.close()


def test_contexts_on_two_streams_take_turns():
    """Two contexts of one loaded library share its constant-memory weight banks.  Driven
    alternately on two streams with no host synchronisation between the calls, each must
    give the losses and state it gives alone: the library orders their passes on the GPU."""
    d1, d2 = config_dict("c2", total_iters=200), config_dict("c1", total_iters=200)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    rgb1, rgb2 = syn.synthetic_image(64, 96, 21), syn.synthetic_image(48, 80, 22)

    def make(d, rgb, H, W, seed, stream):
        cfg = cc.make_config(d, seed=seed)
        init = cc.flatten_params(syn.initial_parameters(syn.ArchSizes.from_config(d), seed), cfg)
        return cc.cc_init_image(cfg, rgb, H, W, init, stream)

    alone = []
    for d, rgb, H, W, seed in ((d1, rgb1, 64, 96, 21), (d2, rgb2, 48, 80, 22)):
        ctx = make(d, rgb, H, W, seed, None)
        try:
            cc.cc_encode_iters(ctx, 40)
            alone.append((cc.cc_get_losses(ctx, 0, 40), cc.cc_get_state(ctx)))
        finally:
            cc.cc_free(ctx)
    a = make(d1, rgb1, 64, 96, 21, s1)
    b = make(d2, rgb2, 48, 80, 22, s2)
    try:
        for _ in range(5):
            cc.cc_encode_iters(a, 8)
            cc.cc_encode_iters(b, 8)
        torch.cuda.synchronize()
        for ctx, (losses, state) in ((a, alone[0]), (b, alone[1])):
            assert np.array_equal(cc.cc_get_losses(ctx, 0, 40), losses)
            assert cc.cc_get_state(ctx) == state
    finally:
        cc.cc_free(a)
        cc.cc_free(b)
