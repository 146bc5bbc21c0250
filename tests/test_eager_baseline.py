"""The PyTorch-eager comparison baseline that bench.py times (its own formulation:
one MLP call over all levels, conv_transpose2d upsampling, torch.optim.Adam) computes the
same iteration as the FP64 oracle: run in float64 on the CPU with the oracle's noise, its
loss, every gradient and the state after Adam steps agree to rounding."""
import numpy as np
import pytest
import torch

from oracle import coolchic as oc
from paper_2403_11651_gb300 import synthetic as syn
from paper_2403_11651_gb300.eager_baseline import EagerIteration, causal_offsets

from .helpers import config_dict, oracle_arch


def _pair(arch, H, W, seed, **kw):
    d = config_dict(arch, **kw)
    init = syn.initial_parameters(syn.ArchSizes.from_config(d), seed)
    rgb = syn.synthetic_image(H, W, seed)
    eager = EagerIteration(rgb, d, init, "cpu", torch.float64)
    enc = oc.OracleEncoder(rgb, oracle_arch(d), oc.Train(lam=d["lam"], lr=d["lr"], seed=seed,
                                                         total_iters=d["total_iters"],
                                                         ste_frac=d["ste_frac"]), init)
    return eager, enc


def _close(a, b, rel):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    assert np.max(np.abs(a - b)) <= rel * max(1.0, float(np.max(np.abs(b)))), \
        float(np.max(np.abs(a - b)))


@pytest.mark.parametrize("n", [8, 16, 24])
def test_causal_offsets_agree(n):
    assert causal_offsets(n) == oc.causal_offsets(n)


@pytest.mark.parametrize("arch,H,W", [("c2", 37, 53), ("c1", 16, 24), ("t300", 67, 45),
                                      ("t545", 20, 33)])
@pytest.mark.parametrize("hard", [False, True])
def test_loss_and_gradients_match_the_oracle(arch, H, W, hard):
    eager, enc = _pair(arch, H, W, 3)
    # a state away from the start: random latents and parameters moved by a few steps
    rng = np.random.default_rng(4)
    ys = [rng.normal(0, 2.0, (h, w)) for h, w in enc.shapes]
    enc.set_latents(ys)
    with torch.no_grad():
        for t, a in zip(eager.y, ys):
            t.copy_(torch.tensor(a))
    u = enc.noise(0)
    L, D, R = eager.loss(noise=u, hard=hard)
    L.backward()
    rL, rD, rR, grads = enc.loss_and_grads(u_levels=None if hard else u, hard=hard)
    assert float(L.detach()) == pytest.approx(rL, rel=1e-12)
    assert float(D.detach()) == pytest.approx(rD, rel=1e-12)
    assert float(R.detach()) == pytest.approx(rR, rel=1e-12)
    mine = [t.grad for t in eager.y] + [eager.P[n].grad for n in enc.names]
    for g, r in zip(mine, grads):
        _close(g.numpy(), r.numpy(), 1e-10)


def test_adam_steps_match_the_oracle():
    eager, enc = _pair("c2", 24, 40, 5, total_iters=6, ste_frac=0.5)
    for t in range(6):                       # three noise steps, then three straight-through
        u = enc.noise(t)
        eager.step(noise=u)
        enc.step(u_levels=u)
    for a, b in zip(eager.y, enc.y):
        _close(a.detach().numpy(), b.detach().numpy(), 1e-9)
    for n in enc.names:
        _close(eager.P[n].detach().numpy(), enc.P[n].detach().numpy(), 1e-9)
