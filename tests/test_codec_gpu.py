"""Latent bitstream on the GPU against the oracle (oracle/codec.py): the bitstream is
bit-exact, the decoded latents are bit-exact, the decoded image is within 0.01 dB PSNR of
the FP64 oracle's decode of the same latents."""
import math

import numpy as np
import pytest
import torch

from oracle import codec as C
from oracle import coolchic as oc
from paper_2403_11651_gb300 import coolchic as cc
from paper_2403_11651_gb300 import synthetic as syn

from .helpers import config_dict, oracle_arch

pytestmark = pytest.mark.gpu


def _decoder_params(d, seed):
    """Seeded float32 decoder parameters with a non-trivial fixed-point ARM."""
    named = syn.initial_parameters(syn.ArchSizes.from_config(d), seed)
    rng = np.random.default_rng(seed + 7)
    for k in named:
        if k.startswith("arm."):
            named[k] = rng.normal(0, 0.15, named[k].shape).astype(np.float32)
    named["arm.bout"] = np.array([0.2, 0.6], np.float32)
    return named


def _latents(H, W, seed, outliers=True, extreme=True):
    """Integer latents, Laplace with a scale growing with the level; escapes planted
    (with extreme: also the largest magnitude the format takes, 2^20)."""
    rng = np.random.default_rng(seed + 11)
    out = []
    for l, s in enumerate(cc.level_shapes(H, W)):
        out.append(np.rint(rng.laplace(0, 0.4 + 0.6 * l, s)).astype(np.int64))
    if outliers:
        if extreme:
            out[0][0, 0] = C.Y_LIM
            out[0][-1, -1] = -C.Y_LIM
        out[1][0, -1] = C.A + 1
        out[2][-1, 0] = -C.A - 1
        out[0][min(3, H - 1), :] = 300
    return out


def _context(d, H, W, named, y):
    cfg = cc.make_config(d, seed=0)
    rgb = syn.synthetic_image(H, W, 3)
    ctx = cc.cc_init_image(cfg, rgb, H, W, cc.flatten_params(named, cfg))
    cc.cc_set_latents(ctx, np.concatenate([a.astype(np.float32).ravel() for a in y]))
    return ctx, rgb


def _psnr(x, ref):
    mse = float(np.mean((np.asarray(x, np.float64) - ref) ** 2))
    return 10 * math.log10(1.0 / mse)


CASES = [("c1", 67, 45, 1), ("c2", 130, 97, 2), ("t1079", 64, 131, 3), ("t300", 33, 70, 4),
         ("c2", 1, 1, 5), ("c1", 9, 300, 6)]


@pytest.mark.parametrize("arch,H,W,seed", CASES)
def test_bitstream_bit_exact(arch, H, W, seed):
    d = config_dict(arch)
    named = _decoder_params(d, seed)
    y = _latents(H, W, seed)
    ctx, _ = _context(d, H, W, named, y)
    try:
        got = cc.cc_write_bitstream(ctx)
        assert cc.cc_write_bitstream(ctx, cc.make_config(d), H, W) == got
        assert len(got) <= cc.bitstream_bound(cc.make_config(d), H, W)
    finally:
        cc.cc_free(ctx)
    want = C.write_bitstream(H, W, oracle_arch(d), named, y)
    assert len(got) == len(want)
    assert got == want


@pytest.mark.parametrize("arch,H,W,seed", CASES)
def test_decode_bit_exact_and_image(arch, H, W, seed):
    d = config_dict(arch)
    arch_o = oracle_arch(d)
    named = _decoder_params(d, seed)
    y = _latents(H, W, seed)
    _, lat, _ = cc.cc_decode_bitstream(C.write_bitstream(H, W, arch_o, named, y), want_rgb=False)
    np.testing.assert_array_equal(lat.astype(np.int64), np.concatenate([a.ravel() for a in y]))
    # image (latents without the 2^20 extremes, which swamp any image error): against the
    # FP64 oracle decode of the same latents and parameters
    y = _latents(H, W, seed, extreme=False)
    bs = C.write_bitstream(H, W, arch_o, named, y)
    rgb, lat, _ = cc.cc_decode_bitstream(bs)
    np.testing.assert_array_equal(lat.astype(np.int64), np.concatenate([a.ravel() for a in y]))
    _, _, _, named2, y2 = C.read_bitstream(bs)
    P = oc.params_from_numpy({k: np.asarray(v, np.float64) for k, v in named2.items()}, arch_o,
                             requires_grad=False)
    with torch.no_grad():
        feat = oc.upsample_all([torch.tensor(a, dtype=oc.DT) for a in y2], P, arch_o,
                               oc.level_shapes(H, W))
        ref = oc.synthesis(feat, P, arch_o).permute(1, 2, 0).numpy()
    x = syn.synthetic_image(H, W, 3).astype(np.float64) / 255.0
    assert abs(_psnr(rgb, x) - _psnr(ref, x)) < 0.01
    assert np.abs(rgb - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_roundtrip_after_training():
    """Overfit a few iterations, code rint(y), decode: latents and image come back, and
    the coded size is the model's rate plus the header and the per-row flush bytes."""
    d = config_dict("c1", total_iters=60)
    H, W = 64, 96
    cfg = cc.make_config(d, seed=0)
    rgb = syn.synthetic_image(H, W, 0)
    ctx = cc.cc_init_image(cfg, rgb, H, W)
    try:
        cc.cc_encode_iters(ctx, 60)
        n_lat = cc.cc_latent_count(cfg, H, W)
        y = np.rint(cc.cc_get_latents(ctx, n_lat)).astype(np.int64)
        img = cc.cc_decode(ctx, H, W)
        _, R, _ = cc.cc_rd_cost(ctx, True)
        bs = cc.cc_write_bitstream(ctx)
    finally:
        cc.cc_free(ctx)
    rgb2, lat, _ = cc.cc_decode_bitstream(bs)
    np.testing.assert_array_equal(lat.astype(np.int64), y)
    np.testing.assert_array_equal(rgb2, img)
    start, streams = C.header_and_streams(bs)
    coded_bits = 8 * sum(len(s) for s in streams)
    model_bits = R * H * W
    rows = len(streams)
    assert coded_bits <= model_bits * 1.05 + 16 * rows
    assert coded_bits >= model_bits * 0.9 - 16 * rows


def test_errors():
    d = config_dict("c1")
    H, W = 16, 16
    named = _decoder_params(d, 0)
    y = _latents(H, W, 0, outliers=False)
    y[0][2, 2] = C.Y_LIM + 1
    ctx, _ = _context(d, H, W, named, y)
    try:
        with pytest.raises(cc.CCError) as e:
            cc.cc_write_bitstream(ctx)
        assert e.value.code == cc.CC_EINVAL
        y[0][2, 2] = 0
        cc.cc_set_latents(ctx, np.concatenate([a.astype(np.float32).ravel() for a in y]))
        import ctypes
        n = ctypes.c_size_t()
        assert cc._lib().cc_write_bitstream(ctx, None, 0, ctypes.byref(n)) == cc.CC_OK
        small = ctypes.create_string_buffer(n.value - 1)
        assert cc._lib().cc_write_bitstream(ctx, small, n.value - 1, ctypes.byref(n)) == cc.CC_ESIZE
        bs = cc.cc_write_bitstream(ctx)
    finally:
        cc.cc_free(ctx)
    # a damaged substream decodes to something or is refused; it never faults
    start, streams = C.header_and_streams(bs)
    body0 = len(bs) - sum(len(s) for s in streams)
    bad = bytearray(bs)
    rng = np.random.default_rng(1)
    for i in rng.integers(body0, len(bs), 16):
        bad[i] ^= 0xFF
    try:
        cc.cc_decode_bitstream(bytes(bad))
    except cc.CCError as e:
        assert e.code == cc.CC_EINVAL
    with pytest.raises(cc.CCError):
        cc.cc_decode_bitstream(bs[:-1])


def test_full_size_2048_c2():
    """2048 x 2048 with the 2300-MAC decoder: sampled substreams bit-exact against the
    oracle, the whole pyramid decodes back exactly, the image within 0.01 dB of FP64."""
    d = config_dict("c2")
    H = W = 2048
    named = _decoder_params(d, 20)
    y = _latents(H, W, 20, extreme=False)
    ctx, _ = _context(d, H, W, named, y)
    try:
        bs = cc.cc_write_bitstream(ctx)
    finally:
        cc.cc_free(ctx)
    arch_o = oracle_arch(d)
    start, streams = C.header_and_streams(bs)
    Q = C.quantize_arm(named, arch_o)
    cum = C.build_tables()
    row0 = np.cumsum([0] + [h for h, _ in cc.level_shapes(H, W)])
    for l, rows in ((0, (0, 1, 3, 1023, 2047)), (1, (0, 511, 1023)), (5, (0, 63)), (6, (0, 31))):
        want = C.encode_rows(y[l], Q, arch_o, cum, rows=rows)
        for r, s in zip(rows, want):
            assert streams[row0[l] + r] == s, (l, r)
    rgb, lat, ms = cc.cc_decode_bitstream(bs)
    np.testing.assert_array_equal(lat.astype(np.int64), np.concatenate([a.ravel() for a in y]))
    P = oc.params_from_numpy({k: np.asarray(v, np.float64) for k, v in named.items()}, arch_o,
                             requires_grad=False)
    with torch.no_grad():
        feat = oc.upsample_all([torch.tensor(a, dtype=oc.DT) for a in y], P, arch_o,
                               oc.level_shapes(H, W))
        ref = oc.synthesis(feat, P, arch_o).permute(1, 2, 0).numpy()
    x = syn.synthetic_image(H, W, 3).astype(np.float64) / 255.0
    assert abs(_psnr(rgb, x) - _psnr(ref, x)) < 0.01
    print(f"2048x2048 c2: {len(bs)} bytes, latent decode {ms:.1f} ms")


def test_decode_on_a_caller_stream():
    """cc_decode_bitstream on a caller's stream (and into device buffers) gives the same
    latents and image as on the default stream."""
    d = config_dict("t1079")
    H, W = 40, 72
    named = _decoder_params(d, 8)
    y = _latents(H, W, 8, extreme=False)
    bs = C.write_bitstream(H, W, oracle_arch(d), named, y)
    rgb0, lat0, _ = cc.cc_decode_bitstream(bs)
    st = torch.cuda.Stream()
    rgb1 = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    lat1 = torch.empty(lat0.shape, dtype=torch.int32, device="cuda")
    cc.cc_decode_bitstream(bs, rgb_out=rgb1, latents_out=lat1, stream=st)
    st.synchronize()
    np.testing.assert_array_equal(lat1.cpu().numpy(), lat0)
    np.testing.assert_array_equal(rgb1.cpu().numpy(), rgb0)


def test_decode_band_wait_gives_up(monkeypatch):
    """Failure detection without a fault: one decoding band never publishes its progress
    (injected on the host); the bands below it give up after their bounded wait, the call
    returns CC_ETIMEOUT, and the next decode on the same device succeeds."""
    d = config_dict("c1")
    H, W = 80, 64                 # level 0: 5 bands of 16 rows
    named = _decoder_params(d, 9)
    y = _latents(H, W, 9, extreme=False)
    bs = C.write_bitstream(H, W, oracle_arch(d), named, y)
    monkeypatch.setenv("CC_DECODE_STALL_BAND", "0")
    monkeypatch.setenv("CC_DECODE_MAX_POLLS", "2000")
    with pytest.raises(cc.CCError) as e:
        cc.cc_decode_bitstream(bs)
    assert e.value.code == cc.CC_ETIMEOUT
    monkeypatch.delenv("CC_DECODE_STALL_BAND")
    monkeypatch.delenv("CC_DECODE_MAX_POLLS")
    _, lat, _ = cc.cc_decode_bitstream(bs, want_rgb=False)
    np.testing.assert_array_equal(lat.astype(np.int64), np.concatenate([a.ravel() for a in y]))
