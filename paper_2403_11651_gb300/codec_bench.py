"""Time the latent bitstream: GPU encode (cc_write_bitstream) and decode
(cc_decode_bitstream) of one image, printed as one JSON line.

    python -m paper_2403_11651_gb300.codec_bench [--config c5] [--iters 0] [--reps 3]

With --iters 0 the pyramid is ``synthetic_latents`` and the decoder its seeded initial
parameters; with --iters n > 0 the context first runs n encoder iterations on the
synthetic image and codes rint of the latents it reached.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import coolchic as cc
from . import synthetic as syn


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c5")
    ap.add_argument("--H", type=int, default=0)
    ap.add_argument("--W", type=int, default=0)
    ap.add_argument("--iters", type=int, default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    d = cc.load_config(a.config)
    H, W = a.H or d["H"], a.W or d["W"]
    cfg = cc.make_config(d, seed=a.seed)
    rgb = syn.synthetic_image(H, W, a.seed)
    ctx = cc.cc_init_image(cfg, rgb, H, W)
    try:
        if a.iters:
            cc.cc_encode_iters(ctx, a.iters)
        else:
            y = syn.synthetic_latents(H, W, a.seed)
            cc.cc_set_latents(ctx, np.concatenate([p.astype(np.float32).ravel() for p in y]))
        enc_ms = []
        for _ in range(a.reps):
            t0 = time.perf_counter()
            bs = cc.cc_write_bitstream(ctx, cfg, H, W)
            enc_ms.append(1e3 * (time.perf_counter() - t0))
    finally:
        cc.cc_free(ctx)
    dec_ms, lat_ms = [], []
    for _ in range(a.reps):
        t0 = time.perf_counter()
        _, _, ms = cc.cc_decode_bitstream(bs, want_latents=False)
        dec_ms.append(1e3 * (time.perf_counter() - t0))
        lat_ms.append(ms)
    n_lat = cc.cc_latent_count(cfg, H, W)
    print(json.dumps({
        "workload": f"{H}x{W} {a.config}, " + (f"{a.iters} encoder iterations" if a.iters
                                                else "synthetic Laplace latents"),
        "bytes": len(bs), "bpp": 8.0 * len(bs) / (H * W), "latents": n_lat,
        "encode_ms": min(enc_ms), "decode_ms": min(dec_ms),
        "latent_decode_ms": min(lat_ms),
        "latent_decode_mlat_per_s": n_lat / (min(lat_ms) * 1e3),
    }))


if __name__ == "__main__":
    main()
