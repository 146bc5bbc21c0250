"""bench.py's algorithmic work counts (the roofline numerators) against the oracle's
decoder MAC count, which is pinned to Table 1 and Fig. 5 (no GPU)."""
import pytest

import bench
from oracle import coolchic as oc
from paper_2403_11651_gb300 import coolchic as cc


def _arch(d):
    return oc.Arch(arm_ctx=d["arm_ctx"], arm_layers=d["arm_layers"], up_kernel=d["up_kernel"],
                   up_per_level=d["up_per_level"], syn_hidden=d["syn_hidden"],
                   syn_res3x3=d["syn_res3x3"])


@pytest.mark.parametrize("name,H,W", [("c2", 512, 768), ("c2", 37, 53), ("c1", 256, 256)])
def test_decoder_macs_match_the_oracle(name, H, W):
    d = cc.load_config(name)
    want = oc.macs_per_pixel(_arch(d), H, W)["total"]
    assert bench.decoder_macs_per_pixel(d, H, W) == pytest.approx(want, rel=1e-12)


def test_arm_flops_per_launch():
    d = cc.load_config("c2")
    n_lat = sum(h * w for h, w in cc.level_shapes(512, 768))
    per_latent = oc.macs_per_pixel(_arch(d), 512, 768)["arm"] * 512 * 768 / n_lat
    # forward, input gradient and weight gradient: three passes of 2 FLOP per MAC
    assert bench.arm_flops_per_launch(d, n_lat) == pytest.approx(6 * per_latent * n_lat, rel=1e-12)
    assert per_latent == pytest.approx(1200) and n_lat == 524256


def test_arm_traffic_tied_to_profiled_sources(monkeypatch):
    """The ARM kernel's DRAM bytes are reported only for the sources they were measured on."""
    monkeypatch.setattr(bench, "ARM_COUNTER_SOURCES_SHA256", bench.arm_sources_sha256())
    assert bench.arm_traffic() == bench.ARM_DRAM_BYTES_PER_LAUNCH
    monkeypatch.setattr(bench, "ARM_COUNTER_SOURCES_SHA256", "0" * 64)
    assert bench.arm_traffic() is None
