"""Short driver for profilers: runs a few overfitting iterations of one configuration.

    python -m paper_2403_11651_gb300.profile --config c2 --warmup 3 --iters 3 [--H h --W w]

Builds a context on the synthetic image, replays `warmup` then `iters` captured iterations
(26 kernels each for the 2300-MAC decoder), then prints the per-phase CUDA-event times of
`--phases` eager iterations.  Kernel launches are therefore: context set-up (2), warm-up,
timed iterations, then the eager phase iterations.
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    from paper_2403_11651_gb300 import coolchic as cc
    from paper_2403_11651_gb300 import synthetic as syn
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c2")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--phases", type=int, default=3)
    ap.add_argument("--H", type=int, default=0)
    ap.add_argument("--W", type=int, default=0)
    ap.add_argument("--timed", type=int, default=0,
                    help="also time this many graph-replayed iterations with CUDA events")
    a = ap.parse_args()
    d = cc.load_config(a.config)
    H, W = a.H or d["H"], a.W or d["W"]
    cfg = cc.make_config(d, seed=0)
    rgb = syn.synthetic_image(H, W, 0)
    init = cc.flatten_params(syn.initial_parameters(syn.ArchSizes.from_config(d), 0), cfg)
    ctx = cc.cc_init_image(cfg, rgb, H, W, init)
    try:
        cc.cc_encode_iters(ctx, a.warmup)
        cc.cc_encode_iters(ctx, a.iters)
        iter_ms = None
        if a.timed:
            import torch
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(torch.cuda.default_stream())
            cc.cc_encode_iters(ctx, a.timed)
            e1.record(torch.cuda.default_stream())
            torch.cuda.synchronize()
            iter_ms = e0.elapsed_time(e1) / a.timed
        ph = cc.cc_profile_phases(ctx, a.phases) if a.phases else []
        D, R, cost = cc.cc_rd_cost(ctx, False)
        print(json.dumps({"H": H, "W": W, "config": a.config,
                          "kernels_per_iteration": cc.cc_graph_kernel_count(ctx),
                          "iter_ms": iter_ms,
                          "phase_ms": {n: float(v) for n, v in zip(cc.PHASES, ph)},
                          "D": D, "R": R, "cost": cost}))
    finally:
        cc.cc_free(ctx)


if __name__ == "__main__":
    main()
