"""GPU test of cc_rate_bits_noalloc, the entry point for callers that cannot allocate
device memory (its scratch is a fixed device array inside the library).

It must give the rate the ordinary path gives -- cc_rd_cost with rint latents, whose R
is bits / (H W) -- within the forward-rate tolerance of the parity tests (rel 1e-5), on
two calls in a row (the second call reuses the scratch the first one left behind).
Collected last, so that a failure here does not stop the rest of the GPU suite.
"""
import numpy as np
import pytest
import torch

from paper_2403_11651_gb300 import coolchic as cc
from paper_2403_11651_gb300 import synthetic as syn

from .helpers import config_dict

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("arch,H,W", [("c2", 512, 768), ("c1", 67, 45), ("t1079", 40, 56)])
def test_noalloc_rate_matches_rd_cost(arch, H, W):
    assert torch.cuda.is_available()
    d = config_dict(arch)
    cfg = cc.make_config(d, seed=5)
    init = cc.flatten_params(syn.initial_parameters(syn.ArchSizes.from_config(d), 5), cfg)
    ctx = cc.cc_init_image(cfg, syn.synthetic_image(H, W, 5), H, W, init)
    try:
        n_lat = cc.cc_latent_count(cfg, H, W)
        rng = np.random.default_rng(5)
        y = rng.normal(0.0, 2.0, n_lat).astype(np.float32)
        cc.cc_set_latents(ctx, y)
        _, R, _ = cc.cc_rd_cost(ctx, True)            # existing entry point, rint latents
        ref_bits = R * H * W
        yhat = torch.from_numpy(np.rint(y)).cuda()
        params = torch.from_numpy(cc.cc_get_params(ctx, cc.cc_param_count(cfg))).cuda()
        first = cc.cc_rate_bits_noalloc(cfg, yhat, H, W, params)
        second = cc.cc_rate_bits_noalloc(cfg, yhat, H, W, params)
        for got in (first, second):
            assert abs(got - ref_bits) <= 1e-5 * ref_bits, (got, ref_bits)
    finally:
        cc.cc_free(ctx)


def test_noalloc_rejects_pyramids_beyond_its_scratch():
    cfg = cc.make_config(config_dict("c2"))
    dummy = torch.zeros(4, device="cuda")
    with pytest.raises(cc.CCError) as e:
        cc.cc_rate_bits_noalloc(cfg, dummy, 4096, 4096, dummy)   # 22.4 M latents
    assert e.value.code == cc.CC_EINVAL
    assert "CC_NOALLOC_MAX_TILES" in cc._lib().cc_last_cuda_error().decode()
