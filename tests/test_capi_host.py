"""C ABI checks that need no GPU: the library builds for sm_103a, loads, exports every
entry point include/coolchic.h declares, and its host-side logic (parameter layout, latent
counts, configuration validation) matches the paper and the binding."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import coolchic as oc
from paper_2403_11651_gb300 import coolchic as cc
from paper_2403_11651_gb300 import synthetic as syn

from .helpers import config_dict

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "coolchic.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(cc_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    return cc.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 20
    raw = ctypes.CDLL(cc.library_path())
    for n in names:
        assert hasattr(raw, n), n
    assert set(names) == set(cc.EXPORTED)


def test_param_count_reproduces_table1(lib, golden_dir):
    import json
    with open(os.path.join(golden_dir, "table1_fig5.json")) as f:
        rows = json.load(f)["table1"]
    for r in rows:
        d = dict(levels=7, arm_ctx=r["arm_ctx"], arm_layers=r["arm_layers"],
                 up_kernel=r["up_kernel"], up_per_level=False, syn_hidden=r["syn_hidden"],
                 syn_res3x3=r["syn_res3x3"], lam=1e-3, lr=1e-2, total_iters=10, ste_frac=0.0)
        assert cc.cc_param_count(cc.make_config(d)) == r["params"]
    assert cc.cc_param_count(cc.make_config(config_dict("c2"))) == 1925 - 64 + 6 * 64


@pytest.mark.parametrize("H,W", [(512, 768), (256, 256), (67, 45), (1, 1), (2048, 2048)])
def test_latent_count(lib, H, W):
    n = cc.cc_latent_count(cc.make_config(config_dict("c2")), H, W)
    assert n == sum(h * w for h, w in oc.level_shapes(H, W))
    if (H, W) == (512, 768):
        assert n == 524256


@pytest.mark.parametrize("field,value", [("levels", 6), ("arm_ctx", 12), ("arm_layers", 3),
                                         ("up_kernel", 6), ("syn_hidden", 32),
                                         ("syn_res3x3", 0), ("ste_frac", 1.5), ("lr", 0.0),
                                         ("total_iters", -1)])
def test_invalid_config_rejected(lib, field, value):
    cfg = cc.make_config(config_dict("c2"))
    setattr(cfg, field, value)
    with pytest.raises(cc.CCError) as e:
        cc.cc_param_count(cfg)
    assert e.value.code == cc.CC_EINVAL


def test_bad_sizes_rejected(lib):
    cfg = cc.make_config(config_dict("c1"))
    for H, W in [(0, 4), (4, 0), (-3, 5)]:
        with pytest.raises(cc.CCError) as e:
            cc.cc_latent_count(cfg, H, W)
        assert e.value.code == cc.CC_EINVAL


def test_strerror(lib):
    assert cc.cc_strerror(0) == "ok"
    for code in (-1, -2, -3, -4, -5, -6, -7):
        assert cc.cc_strerror(code) != "unknown error"
    assert cc.cc_strerror(-99) == "unknown error"


@pytest.mark.parametrize("arch", ["c1", "c2", "t300", "t1079"])
def test_binding_layout_matches_oracle_order(arch):
    d = config_dict(arch)
    cfg = cc.make_config(d)
    a = oc.Arch(arm_ctx=d["arm_ctx"], arm_layers=d["arm_layers"], up_kernel=d["up_kernel"],
                up_per_level=d["up_per_level"], syn_hidden=d["syn_hidden"],
                syn_res3x3=d["syn_res3x3"])
    assert cc.param_layout(cfg) == [(n, tuple(s)) for n, s in oc.param_shapes(a)]
    init = syn.initial_parameters(syn.ArchSizes.from_config(d), 3)
    flat = cc.flatten_params(init, cfg)
    back = cc.unflatten_params(flat, cfg)
    for k in init:
        assert np.array_equal(back[k], init[k])


def test_config_files_load():
    for name in ("c1", "c2", "c5"):
        d = cc.load_config(name)
        cfg = cc.make_config(d)
        assert cfg.levels == 7 and cfg.total_iters == d["total_iters"]


@pytest.mark.parametrize("arch,H,W", [("c1", 37, 53), ("t1079", 5, 300)])
def test_bitstream_header_parsed_on_host(lib, arch, H, W):
    """cc_bitstream_info reads an oracle-written bitstream; damaged or truncated streams are
    refused on the host, before any device work."""
    from oracle import codec as C
    from .helpers import oracle_arch
    d = config_dict(arch)
    a = oracle_arch(d)
    rng = np.random.default_rng(0)
    named = {n: rng.normal(0, 0.1, s).astype(np.float32) for n, s in oc.param_shapes(a)}
    y = [np.rint(rng.laplace(0, 1.0, s)).astype(np.int64) for s in oc.level_shapes(H, W)]
    bs = C.write_bitstream(H, W, a, named, y)
    cfg, h, w = cc.cc_bitstream_info(bs)
    assert (h, w) == (H, W)
    got = (cfg.levels, cfg.arm_ctx, cfg.arm_layers, cfg.up_kernel, cfg.up_per_level,
           cfg.syn_hidden, cfg.syn_res3x3)
    assert got == (7, d["arm_ctx"], d["arm_layers"], d["up_kernel"], int(d["up_per_level"]),
                   d["syn_hidden"], d["syn_res3x3"])
    for bad in (b"XXXX" + bs[4:], bs[:-1], bs + b"\0", bs[:30]):
        with pytest.raises(cc.CCError) as e:
            cc.cc_decode_bitstream(bad)
        assert e.value.code == cc.CC_EINVAL
    wrong_arch = bytearray(bs)
    wrong_arch[13] = 7          # N = 7 is not a supported context size
    with pytest.raises(cc.CCError):
        cc.cc_bitstream_info(bytes(wrong_arch))


@pytest.mark.parametrize("arch,H,W", [("c1", 1, 1), ("c2", 33, 47), ("t300", 64, 9)])
def test_bitstream_bound_holds(lib, arch, H, W):
    """The binding's output-buffer bound covers bitstreams of extreme latents (escapes of
    2^20 everywhere)."""
    from oracle import codec as C
    from .helpers import oracle_arch
    d = config_dict(arch)
    a = oracle_arch(d)
    rng = np.random.default_rng(1)
    named = {n: rng.normal(0, 0.1, s).astype(np.float32) for n, s in oc.param_shapes(a)}
    y = [np.where(rng.random(s) < 0.5, C.Y_LIM, -C.Y_LIM).astype(np.int64)
         for s in oc.level_shapes(H, W)]
    bs = C.write_bitstream(H, W, a, named, y)
    assert len(bs) <= cc.bitstream_bound(cc.make_config(d), H, W)


def test_library_copies_load_independently(lib):
    """The batch runner's lanes are separately loaded copies of the library, each its own
    module (and so its own constant banks); each answers through the C ABI."""
    import ctypes
    from paper_2403_11651_gb300.batch import library_instances
    libs = library_instances(3)
    assert len({l._handle for l in libs}) == 3
    cfg = cc.make_config(config_dict("c2"))
    for l in libs:
        n = ctypes.c_int()
        assert l.cc_param_count(ctypes.byref(cfg), ctypes.byref(n)) == 0
        assert n.value == cc.cc_param_count(cfg)


def test_warm_predictor_host_checks(lib):
    """Parameter count of the warm-start predictor (4 convolutions of 32 channels, 5
    heads) and its argument checks, all taken before any device work."""
    ch = 32
    want = (ch * 3 * 9 + ch) + 3 * (ch * ch * 9 + ch) + 4 * (ch + 1) + (3 * 9 + 1)
    assert cc.cc_warm_param_count() == want == 28800
    params = np.zeros(want, np.float32)
    for H, W in [(15, 64), (64, 15), (16385, 64), (0, 0)]:
        with pytest.raises(cc.CCError) as e:
            cc.cc_warm_create(H, W, params)
        assert e.value.code == cc.CC_EINVAL
    assert lib.cc_warm_predict(None, None, None) == cc.CC_EINVAL
    assert lib.cc_warm_set_params(None, None) == cc.CC_EINVAL
    lib.cc_warm_free(None)
