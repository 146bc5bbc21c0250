"""Learned warm start against plain overfitting, printed as one JSON line.

    python -m paper_2403_11651_gb300.warm_bench [--train 48] [--test 8] [--iters 1000]
        [--size 256] [--test-size H W] [--ablate K] [--max-data-s S]

1. This project's encoder overfits --train synthetic --size x --size images (2300-MAC
   decoder, --iters iterations, all from one seeded initial decoder; --chunk at a time
   through the batch runner, stopping early once --max-data-s seconds have been spent):
   the pairs (image, latents reached) and the decoders reached.
2. The warm-start predictor (cc_warm_*) is trained on those pairs (Adam, --epochs).
3. On --test held-out images of --test-size (default: the training size; a second
   predictor of that size takes the trained parameters): the plain method (latents 0,
   the same seeded initial decoder) and the warm start (predicted latents, the mean of the
   trained decoders) run the same schedule (--iters iterations, the last 20 %
   straight-through); the hard RD cost is read every --every iterations.  Reported: the
   warm start's iterations and seconds to reach the plain run's final RD cost within 1 %,
   and both final RD costs; on the first --ablate held-out images also the mean decoder
   alone and the predicted latents alone.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

from .batch import BatchOverfitter   # first: sets the hardware queue count before CUDA starts
from . import coolchic as cc
from . import synthetic as syn


def config(iters: int):
    d = dict(cc.load_config("c2"))
    d["total_iters"] = iters
    return d


def checkpoints(iters: int, every: int):
    """Iteration counts at which run_schedule reads the cost: 0, every, 2 every, ..., iters."""
    out = list(range(0, iters, every)) + [iters]
    return out if iters > 0 else [0]


def first_at_or_below(curve, target):
    """Index of the first entry of curve at or below target, or None."""
    hit = np.nonzero(np.asarray(curve) <= target)[0]
    return int(hit[0]) if hit.size else None


def run_schedule(cfg, rgb, init_params, latents, iters, every):
    """Hard RD cost at each of checkpoints(iters, every), and the seconds spent up to each
    (host clock around the iterations and the synchronising cost reads; 0 at the start)."""
    H, W = rgb.shape[:2]
    ctx = cc.cc_init_image(cfg, rgb, H, W, init_params)
    try:
        if latents is not None:
            cc.cc_set_latents(ctx, latents)
        costs = [cc.cc_rd_cost(ctx, True)[2]]
        spent = 0.0
        secs = [0.0]
        done = 0
        while done < iters:
            n = min(every, iters - done)
            t0 = time.perf_counter()
            cc.cc_encode_iters(ctx, n)
            cc.cc_iteration(ctx)
            c = cc.cc_rd_cost(ctx, True)[2]      # synchronises
            spent += time.perf_counter() - t0
            costs.append(c)
            secs.append(spent)
            done += n
        return np.array(costs), np.array(secs)
    finally:
        cc.cc_free(ctx)


def batched_eval(a, d, init, dec, starts, plain_finals):
    """The held-out images as one batch on a.lanes concurrent lanes (every image's
    iterations bit-identical to its own run).  Plain: zero latents and the seeded decoder
    for the whole schedule.  Warm: the predicted latents and the mean trained decoder until
    every image's hard RD cost is within 1 % of its plain run's final cost, read every
    a.every iterations.  Plain runs the whole schedule (the runner synchronises every
    a.every iterations) and reads the costs once at the end.  Seconds on the host clock
    from the first iteration; the warm start's include the predictor's inference of every
    image."""
    cps = checkpoints(a.iters, a.every)

    def run(init_params, latents, targets):
        items = [(rgb, d, init_params, a.train + j) for j, (rgb, _, _, _) in enumerate(starts)]
        b = BatchOverfitter(items, lanes=a.lanes, chunk=16)
        try:
            if latents is not None:
                for i, y in enumerate(latents):
                    b.set_latents(i, y)
            reached = [None] * len(items)
            done = 0
            t0 = time.perf_counter()
            for it in cps[1:]:
                b.run(it - done)
                done = it
                if targets is None:
                    continue
                for i, (_, _, cost) in enumerate(b.rd_costs()):
                    if reached[i] is None and cost <= targets[i]:
                        reached[i] = it
                if all(r is not None for r in reached):
                    break
            if targets is None:
                b.rd_costs()
            return time.perf_counter() - t0, reached, done
        finally:
            b.close()

    t_plain, _, _ = run(init, None, None)
    targets = [p * 1.01 for p in plain_finals]
    t_warm, reached, stopped = run(dec, [y for _, _, y, _ in starts], targets)
    t_pred = sum(t for _, _, _, t in starts)
    return {"images": len(starts), "lanes": a.lanes,
            "plain_batched_s": t_plain,
            "warm_batched_s_to_all_reached": t_warm + t_pred,
            "warm_stopped_at_iter": stopped,
            "warm_reached_iters": reached,
            "all_reached": all(r is not None for r in reached)}


def parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=48)
    ap.add_argument("--test", type=int, default=8)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--iters", type=int, default=1000)
    ap.add_argument("--every", type=int, default=25)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--test-size", type=int, nargs=2, default=None, metavar=("H", "W"))
    ap.add_argument("--ablate", type=int, default=None)
    ap.add_argument("--chunk", type=int, default=64)
    ap.add_argument("--max-data-s", type=float, default=float("inf"))
    ap.add_argument("--batched-eval", action="store_true",
                    help="also run the held-out images as one batch (concurrent lanes): "
                         "plain for the whole schedule, and warm-started until every image "
                         "reaches its plain run's final cost")
    ap.add_argument("--lanes", type=int, default=8)
    ap.add_argument("--step-time", action="store_true",
                    help="only time the predictor's training step at --size (inputs in device "
                         "memory, the loss written to device memory)")
    return ap


def step_time(S: int, steps: int = 200, warmup: int = 10) -> dict:
    """Device time per training step of the predictor on one S x S image: image, target and
    loss in device memory, CUDA events around `steps` queued steps."""
    import torch
    n_lat = sum(h * w for h, w in cc.level_shapes(S, S))
    rgb = torch.from_numpy(syn.synthetic_image(S, S, 1)).cuda()
    tgt = torch.from_numpy(np.random.default_rng(1).normal(0, 1.0, n_lat)
                           .astype(np.float32)).cuda()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    w = cc.cc_warm_create(S, S, syn.warm_initial_parameters(1), stream)
    try:
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                cc.cc_warm_train_step(w, rgb, tgt, 1e-3, loss_out=loss)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                cc.cc_warm_train_step(w, rgb, tgt, 1e-3, loss_out=loss)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        gflop = 2.0 * warm_macs_per_step(S) / 1e9
        return {"size": S, "step_ms": ms, "gflop_per_step": gflop,
                "tflops": gflop / ms, "loss": float(loss.cpu()[0])}
    finally:
        cc.cc_warm_free(w)


def warm_macs_per_step(S: int) -> int:
    """Multiply-adds of one training step at S x S: conv 1 forward and weight gradient,
    conv 2 .. 4 forward, input and weight gradients, head 0 forward and weight gradient,
    heads 1 .. 4 forward, weight and input gradients."""
    h = [S]
    for _ in range(4):
        h.append((h[-1] + 1) // 2)
    px = [x * x for x in h]
    macs = 2 * px[1] * 32 * 27                      # conv 1: forward, weight gradient
    macs += sum(3 * px[i] * 32 * 288 for i in (2, 3, 4))
    macs += 2 * px[0] * 27                          # head 0
    macs += sum(3 * px[i] * 32 for i in (1, 2, 3, 4))
    return macs


def main(argv=None):
    a = parser().parse_args(argv)
    if a.step_time:
        print(json.dumps(step_time(a.size)))
        return
    # the synthetic images are made on the host cores while the GPU overfits (a spawned
    # pool, started before this process's first CUDA call)
    pool = ProcessPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) - 2)),
                               mp_context=mp.get_context("spawn"))
    try:
        print(json.dumps(experiment(a, pool)))
    finally:
        pool.shutdown(cancel_futures=True)


def experiment(a, pool):
    """The whole experiment for the options a (see parser()); pool makes the synthetic
    images (anything with submit(fn, *args) -> future)."""
    S = a.size
    TH, TW = a.test_size if a.test_size else (S, S)
    n_ablate = a.test if a.ablate is None else min(a.ablate, a.test)
    d = config(a.iters)
    n_params = cc.cc_param_count(cc.make_config(d))
    # one seeded initial decoder for every run: decoders trained from different random
    # starts differ by a permutation of their hidden units, so only decoders that share a
    # start have a meaningful mean (measured: with one start per image the mean of 1792
    # decoders left the warm runs at 6.6x the plain RD cost), and the latents they reach
    # are consistent enough across images to be predicted
    init = cc.flatten_params(syn.initial_parameters(syn.ArchSizes.from_config(d), 0),
                             cc.make_config(d))

    train_img = [pool.submit(syn.synthetic_image, S, S, 1000 + k) for k in range(a.train)]
    test_img = [pool.submit(syn.synthetic_image, TH, TW, 1000 + k)
                for k in range(a.train, a.train + a.test)]

    # 1. training pairs from this project's own encoder
    t0 = time.perf_counter()
    images, lat, dec_sum = [], [], np.zeros(n_params, np.float64)
    for c0 in range(0, a.train, a.chunk):
        if time.perf_counter() - t0 > a.max_data_s:
            break
        items = [(train_img[k].result(), d, init, k)
                 for k in range(c0, min(a.train, c0 + a.chunk))]
        b = BatchOverfitter(items, lanes=8)
        try:
            b.run(a.iters)
            lat += [b.latents(i) for i in range(len(items))]
            for i in range(len(items)):
                dec_sum += b.params(i, n_params)
        finally:
            b.close()
        images += [it[0] for it in items]
    n_train = len(images)
    dec = (dec_sum / n_train).astype(np.float32)
    t_data = time.perf_counter() - t0

    # 2. the predictor: training pairs resident in device memory, one loss per step written
    # to device memory, read once per epoch
    import torch
    w = cc.cc_warm_create(S, S, syn.warm_initial_parameters(0))
    wt = None
    try:
        d_img = torch.from_numpy(np.stack(images)).cuda()
        d_lat = torch.from_numpy(np.stack(lat)).cuda()
        d_loss = torch.zeros(n_train, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        losses = []
        order = np.random.default_rng(0)
        for ep in range(a.epochs):
            for i in order.permutation(n_train):
                cc.cc_warm_train_step(w, d_img[i], d_lat[i], a.lr, loss_out=d_loss[i])
            losses.append(float(d_loss.mean()))
            if not np.isfinite(losses[-1]):
                raise RuntimeError(f"predictor loss not finite in epoch {ep}")
        t_train = time.perf_counter() - t0
        t_step_ms = t_train / max(1, a.epochs * n_train) * 1e3
        if (TH, TW) == (S, S):
            wt = w
        else:
            wt = cc.cc_warm_create(TH, TW, cc.cc_warm_get_params(w))

        # 3. held-out images: plain against warm start
        n_lat = sum(h * w_ for h, w_ in cc.level_shapes(TH, TW))
        res, curves, starts = [], [], []
        for j, k in enumerate(range(a.train, a.train + a.test)):
            rgb = test_img[j].result()
            cfg = cc.make_config(d, seed=k)
            t0 = time.perf_counter()
            y0 = cc.cc_warm_predict(wt, rgb, n_lat)
            t_pred = time.perf_counter() - t0
            starts.append((rgb, cfg, y0, t_pred))
            plain, plain_s = run_schedule(cfg, rgb, init, None, a.iters, a.every)
            warm, warm_s = run_schedule(cfg, rgb, dec, y0, a.iters, a.every)
            # ablations: the mean decoder alone (latents 0), the predicted latents alone
            if j < n_ablate:
                dec_only, _ = run_schedule(cfg, rgb, dec, None, a.iters, a.every)
                lat_only, _ = run_schedule(cfg, rgb, init, y0, a.iters, a.every)
            target = plain[-1] * 1.01
            cps = checkpoints(a.iters, a.every)

            def first_hit(curve):
                i = first_at_or_below(curve, target)
                return cps[i] if i is not None else None
            i_hit = first_at_or_below(warm, target)
            it_hit = cps[i_hit] if i_hit is not None else None
            curves.append((plain / plain[-1], warm / plain[-1]))
            res.append({"plain_final": float(plain[-1]), "warm_final": float(warm[-1]),
                        "plain_start": float(plain[0]), "warm_start": float(warm[0]),
                        "warm_iters_to_plain_final": it_hit,
                        "decoder_only_iters_to_plain_final":
                            first_hit(dec_only) if j < n_ablate else "not run",
                        "latents_only_iters_to_plain_final":
                            first_hit(lat_only) if j < n_ablate else "not run",
                        "warm_s_to_plain_final": (t_pred + float(warm_s[i_hit]))
                        if i_hit is not None else None,
                        "plain_s": float(plain_s[-1])})
    finally:
        if wt is not None and wt is not w:
            cc.cc_warm_free(wt)
        cc.cc_warm_free(w)
    batched = batched_eval(a, d, init, dec, starts, [r["plain_final"] for r in res]) \
        if a.batched_eval else None
    hits = [r["warm_iters_to_plain_final"] for r in res]

    def mean_hits(key):
        h = [r[key] for r in res if r[key] != "not run"]
        if not h:
            return (None, 0)
        return (float(np.mean([x if x is not None else a.iters for x in h])),
                sum(x is not None for x in h))
    cps = checkpoints(a.iters, a.every)
    pick = list(range(0, len(cps), 4))
    if pick[-1] != len(cps) - 1:
        pick.append(len(cps) - 1)
    return {
        "workload": f"{n_train} training synthetic {S}x{S} / {a.test} held-out synthetic "
                    f"{TH}x{TW} images, 2300-MAC decoder, {a.iters} iterations (last 20 % "
                    f"straight-through); ablations on {n_ablate} held-out images",
        "train_requested": a.train, "epochs": a.epochs, "lr": a.lr,
        "data_s": t_data, "predictor_train_s": t_train, "predictor_step_ms": t_step_ms,
        "predictor_loss_first_last_epoch": [losses[0], losses[-1]],
        "reached": sum(h is not None for h in hits), "of": len(hits),
        "mean_iters_to_plain_final": float(np.mean([h for h in hits if h is not None]))
        if any(h is not None for h in hits) else None,
        "ablation_mean_iters_reached": {
            "predicted_latents_and_mean_decoder": mean_hits("warm_iters_to_plain_final"),
            "mean_decoder_only": mean_hits("decoder_only_iters_to_plain_final"),
            "predicted_latents_only": mean_hits("latents_only_iters_to_plain_final")},
        "mean_plain_s": float(np.mean([r["plain_s"] for r in res])),
        "mean_warm_s_to_plain_final_reached": float(np.mean(
            [r["warm_s_to_plain_final"] for r in res if r["warm_s_to_plain_final"] is not None]))
        if any(r["warm_s_to_plain_final"] is not None for r in res) else None,
        "curve_iters": [cps[i] for i in pick],
        "mean_cost_over_plain_final": {
            "plain": [float(v) for v in np.mean([c[0] for c in curves], axis=0)[pick]],
            "warm": [float(v) for v in np.mean([c[1] for c in curves], axis=0)[pick]]},
        "mean_final_cost_ratio_warm_over_plain": float(np.mean(
            [r["warm_final"] / r["plain_final"] for r in res])),
        "mean_start_cost_ratio_warm_over_plain": float(np.mean(
            [r["warm_start"] / r["plain_start"] for r in res])),
        "batched_eval": batched,
        "per_image": res}


if __name__ == "__main__":
    main()
