"""Batched overfitting of many images of uneven sizes against running them one after the
other, printed as one JSON line.

    python -m paper_2403_11651_gb300.batch_bench [--images 32] [--iters 300] [--lanes 8]
                                                 [--max-pixels N] [--autotune] [--small t300]

Workload: images of sizes drawn uniformly from 256x256, 512x768, 768x512, 1024x1024 and
1920x1080 (seeded synthetic images), half with the first configuration's decoder and half
with the 2300-MAC one, lambda log-uniform in [1e-4, 1e-2].  Both runs start from the
same state and run the same iterations: the final RD costs must agree exactly.  With
--autotune the lane count and chunk length come from batch.autotune instead of --lanes.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from .batch import BatchOverfitter, autotune   # first: sets the hardware queue count
from . import coolchic as cc
from . import synthetic as syn

SIZES = [(256, 256), (512, 768), (768, 512), (1024, 1024), (1080, 1920)]


def workload(n: int, seed: int, max_pixels: int = 0, small: str = "c1"):
    """n seeded images: sizes uniform over SIZES (at most max_pixels each), even-numbered
    images with the decoder of configuration `small`, odd ones with the 2300-MAC one."""
    rng = np.random.default_rng(seed)
    sizes = [s for s in SIZES if not max_pixels or s[0] * s[1] <= max_pixels]
    items = []
    for k in range(n):
        H, W = sizes[int(rng.integers(len(sizes)))]
        d = dict(cc.load_config(small if k % 2 == 0 else "c2"))
        d["lam"] = float(math.exp(rng.uniform(math.log(1e-4), math.log(1e-2))))
        cfg = cc.make_config(d, seed=k)
        init = cc.flatten_params(syn.initial_parameters(syn.ArchSizes.from_config(d), k), cfg)
        items.append((syn.synthetic_image(H, W, k), d, init, k))
    return items


def timed(items, lanes, iters, chunk=16):
    b = BatchOverfitter(items, lanes=lanes, chunk=chunk)
    try:
        b.run(3)                              # graph capture and warm-up
        t0 = time.perf_counter()
        b.run(iters)
        dt = time.perf_counter() - t0
        return dt, b.rd_costs()
    finally:
        b.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--images", type=int, default=32)
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--lanes", type=int, default=8)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--max-pixels", type=int, default=0,
                    help="only the sizes with at most this many pixels (0: all)")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--small", default="c1",
                    help="configuration of the even-numbered images' decoder (c1: the first "
                         "configuration; t300: Table 1's 300-MAC row)")
    a = ap.parse_args(argv)
    items = workload(a.images, a.seed, a.max_pixels, a.small)
    sizes = [s for s in SIZES if not a.max_pixels or s[0] * s[1] <= a.max_pixels]
    px = sum(rgb.shape[0] * rgb.shape[1] for rgb, _, _, _ in items)
    lanes, chunk, tune = a.lanes, 16, None
    if a.autotune:
        t0 = time.perf_counter()
        (lanes, chunk), table = autotune(items)
        tune = {"seconds": time.perf_counter() - t0,
                "probe_s": {f"{k[0]}x{k[1]}": v for k, v in table.items()}}
    t_plain, rd_plain = timed(items, 1, a.iters)
    t_batch, rd_batch = timed(items, lanes, a.iters, chunk)
    small = [i for i, (rgb, _, _, _) in enumerate(items) if rgb.shape[0] * rgb.shape[1] <= 512 * 768]
    print(json.dumps({
        "workload": f"{a.images} images ({px / 1e6:.1f} Mpixel), sizes in {sizes}, "
                    f"half {a.small} / half 2300-MAC decoders, lambda log-uniform "
                    f"[1e-4, 1e-2], {a.iters} iterations each",
        "plain_s": t_plain, "batched_s": t_batch, "lanes": lanes, "chunk": chunk,
        "autotune": tune,
        "speedup": t_plain / t_batch,
        "plain_mpx_iter_s": px * a.iters / t_plain / 1e6,
        "batched_mpx_iter_s": px * a.iters / t_batch / 1e6,
        "final_rd_identical": rd_plain == rd_batch,
        "images_at_most_512x768": len(small),
    }))


if __name__ == "__main__":
    main()
