"""Kernel-start timeline of one replayed overfitting iteration (traced library build).

    python -m paper_2403_11651_gb300.trace [--config c2] [--warmup 30] [--iters 4] [--all]

Builds _build/libcoolchic_trace.so (build.py --trace), creates a context on the synthetic
image of the configuration, replays `warmup` captured iterations, clears the trace, replays
`iters` more and prints, for the second of them (every one with --all), the start time of
each kernel's first block relative to the iteration's first kernel and the time to the
next start.  Kernels of the side stream (the ARM kernel and the context gather) appear in
start order among those of the chain.  The timer is the GPU's global timer; the records are
taken after each kernel's dependency wait.
"""
import argparse
import ctypes
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KERNELS = ["k_arm_fb", "k_arm_fwd", "k_arm_image", "k_syn_image", "k_quantize", "k_up_fwd", "k_up_bwd",
           "k_syn1x1_fwd", "k_syn1x1_bwd", "k_conv3_fwd", "k_conv3_last", "k_conv3_mid", "k_conv3_pair",
           "k_ctx_gather", "k_reduce_sections", "k_param_update", "k_latent_update", "k_finish",
           "k_image_to_planar", "k_planar_to_hwc", "k_rate_noalloc", "k_sum_tiles",
           "finish_begin", "finish_end", "param_block_done"]


class TraceRec(ctypes.Structure):
    _fields_ = [("t", ctypes.c_ulonglong), ("hash", ctypes.c_uint), ("gx", ctypes.c_int),
                ("gy", ctypes.c_int), ("bx", ctypes.c_int)]


def fnv1a(name: str) -> int:
    h = 2166136261
    for ch in name.encode():
        h = ((h ^ ch) * 16777619) & 0xFFFFFFFF
    return h


def main():
    from paper_2403_11651_gb300 import build as _build
    from paper_2403_11651_gb300 import coolchic as cc
    from paper_2403_11651_gb300 import synthetic as syn
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c2")
    ap.add_argument("--warmup", type=int, default=30)
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--all", action="store_true")
    a = ap.parse_args()
    lib = cc._declare(ctypes.CDLL(_build.build_trace()))
    lib.cc_trace_dump.restype = ctypes.c_int
    lib.cc_trace_dump.argtypes = [ctypes.c_void_p, ctypes.c_int]
    cc._LIB = lib
    names = {fnv1a(n): n for n in KERNELS}

    d = cc.load_config(a.config)
    H, W = d["H"], d["W"]
    cfg = cc.make_config(d, seed=0)
    rgb = syn.synthetic_image(H, W, 0)
    init = cc.flatten_params(syn.initial_parameters(syn.ArchSizes.from_config(d), 0), cfg)
    ctx = cc.cc_init_image(cfg, rgb, H, W, init)
    try:
        buf = (TraceRec * 8192)()
        cc.cc_encode_iters(ctx, a.warmup)
        lib.cc_trace_dump(ctypes.addressof(buf), 8192)
        cc.cc_encode_iters(ctx, a.iters)
        n = lib.cc_trace_dump(ctypes.addressof(buf), 8192)
    finally:
        cc.cc_free(ctx)
    recs = sorted((buf[i].t, names.get(buf[i].hash, hex(buf[i].hash)), buf[i].gx, buf[i].gy,
                   buf[i].bx) for i in range(min(n, 8192)))
    starts = [i for i, r in enumerate(recs) if r[1] == "k_quantize"]
    print(f"{a.config} {H}x{W}: {n} kernel records, {len(starts)} iterations")
    for idx, (s0, s1) in enumerate(zip(starts, starts[1:])):
        if idx != 1 and not a.all:
            continue
        seg, t_next = recs[s0:s1], recs[s1][0]
        tb = seg[0][0]
        print(f"--- iteration {idx}: {(t_next - tb) / 1e3:.2f} us")
        for j, r in enumerate(seg):
            nxt = seg[j + 1][0] if j + 1 < len(seg) else t_next
            print(f"  {(r[0] - tb) / 1e3:8.2f}  +{(nxt - r[0]) / 1e3:7.2f}  {r[1]:18s} "
                  f"grid {r[2]}x{r[3]} block {r[4]}")


if __name__ == "__main__":
    main()
