"""GPU test of cc_rate_bits_noalloc, the entry point for callers that cannot allocate
device memory: a decoder inside a process whose device memory is all owned by another
allocator, or a real-time service that must not allocate once running.  Its scratch is a
fixed device array inside the library.

It must give the rate the ordinary path gives -- cc_rd_cost with rint latents, whose R
is bits / (H W) -- and the FP64 oracle's total bits, within the forward-rate tolerance of
the parity tests (rel 1e-5), on two calls in a row (the second call reuses the scratch
the first one left behind), on the legacy default stream and on a caller's stream, with
the total written to host or to device memory.  The first call is the warm-up its header
asks for; the device's free memory must not change across the second.  Collected last,
so that a failure here does not stop the rest of the GPU suite.
"""
import numpy as np
import pytest
import torch

from oracle import coolchic as oc
from paper_2403_11651_gb300 import coolchic as cc
from paper_2403_11651_gb300 import synthetic as syn

from .helpers import config_dict, oracle_arch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("arch,H,W,on_stream,to_device",
                         [("c2", 512, 768, False, False), ("c2", 512, 768, True, True),
                          ("c1", 67, 45, True, False), ("t1079", 40, 56, False, True)])
def test_noalloc_rate_matches_rd_cost(arch, H, W, on_stream, to_device):
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
        prm_host = cc.cc_get_params(ctx, cc.cc_param_count(cfg))
        yhat = torch.from_numpy(np.rint(y)).cuda()
        params = torch.from_numpy(prm_host).cuda()
        stream = torch.cuda.Stream() if on_stream else None
        outs = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(2)] \
            if to_device else [None, None]
        torch.cuda.synchronize()
        got = [cc.cc_rate_bits_noalloc(cfg, yhat, H, W, params, stream, outs[0])]
        free_before = torch.cuda.mem_get_info()[0]
        got.append(cc.cc_rate_bits_noalloc(cfg, yhat, H, W, params, stream, outs[1]))
        free_after = torch.cuda.mem_get_info()[0]
        assert free_after == free_before, (free_before, free_after)
        if to_device:
            got = [float(o.cpu()[0]) for o in got]
        # the FP64 oracle's rate of the same rounded pyramid and ARM parameters (eq. (1) R)
        levels = [torch.from_numpy(a.astype(np.float64))
                  for a in cc.split_latents(np.rint(y), H, W)]
        P = oc.params_from_numpy(cc.unflatten_params(prm_host, cfg), oracle_arch(d),
                                 requires_grad=False)
        oracle_bits = float(oc.total_bits(levels, P, oracle_arch(d)))
        for g in got:
            assert abs(g - ref_bits) <= 1e-5 * ref_bits, (g, ref_bits)
            assert abs(g - oracle_bits) <= 1e-5 * oracle_bits, (g, oracle_bits)
    finally:
        cc.cc_free(ctx)


def test_noalloc_rejects_pyramids_beyond_its_scratch():
    cfg = cc.make_config(config_dict("c2"))
    dummy = torch.zeros(4, device="cuda")
    with pytest.raises(cc.CCError) as e:
        cc.cc_rate_bits_noalloc(cfg, dummy, 4096, 4096, dummy)   # 22.4 M latents
    assert e.value.code == cc.CC_EINVAL
    assert "CC_NOALLOC_MAX_TILES" in cc._lib().cc_last_cuda_error().decode()
