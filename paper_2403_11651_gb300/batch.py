"""Several images overfitted at once (argument marshalling and scheduling only; every
iteration runs in the CUDA library).

The decoder weights of a context live in the library's ``__constant__`` banks, which all
contexts of one loaded library share, so the library runs their passes one after another
on the GPU.  Each separately loaded copy of the shared library registers its own device
module and so owns its own banks, and contexts of different copies run concurrently.  ``BatchOverfitter`` deals the images to ``lanes`` copies: lane i's images
take turns on the lane's stream (``chunk`` iterations each), and the lanes run
concurrently -- small, latency-bound images then share the GPU instead of each leaving it
mostly idle.  Every image runs exactly the iterations it would run alone (same kernels,
same state, its own weights and schedule), so its results are bit-identical.
``autotune`` picks the lane count and chunk length for a batch by timing each candidate
on throwaway contexts of the same images.
"""
from __future__ import annotations

import ctypes
import os
import shutil

import numpy as np

from . import build as _build
from . import coolchic as cc

# CUDA maps streams onto a fixed number of hardware work queues (8 by default); the lanes'
# streams and each context's side stream need more, or the lanes serialise behind one
# another (measured: 8 lanes of 256 x 256 images 3x faster with 32 queues, no change for
# one lane).  Only effective before the process's first CUDA call: import this module
# first, or set the variable in the environment.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

INSTANCE_DIR = os.path.join(_build.BUILD, "instances")


def library_instances(k: int):
    """k independently loaded copies of the library (the built one first)."""
    cc.load()
    libs = [cc._lib()]
    os.makedirs(INSTANCE_DIR, exist_ok=True)
    for i in range(1, k):
        path = os.path.join(INSTANCE_DIR, f"libcoolchic_{i}.so")
        if (not os.path.exists(path)
                or os.path.getmtime(path) < os.path.getmtime(_build.LIB)
                or os.path.getsize(path) != os.path.getsize(_build.LIB)):
            tmp = path + ".tmp"
            shutil.copy2(_build.LIB, tmp)
            os.replace(tmp, path)
        libs.append(cc._declare(ctypes.CDLL(path)))
    return libs


def _check(lib, code: int, where: str):
    if code != cc.CC_OK:
        raise RuntimeError(f"{where}: {lib.cc_strerror(code).decode()} ({code}): "
                           f"{lib.cc_last_cuda_error().decode()}")


class BatchOverfitter:
    """items: (rgb uint8 H x W x 3, configuration dict of configs/*.json or cc_config,
    flat initial parameters or None, seed); lanes: library copies run concurrently."""

    def __init__(self, items, lanes: int = 8, chunk: int = 16):
        import torch
        self.lanes = max(1, min(lanes, len(items)))
        self.chunk = chunk
        self.libs = library_instances(self.lanes)
        self.streams = [torch.cuda.Stream() for _ in range(self.lanes)]
        self.ctx, self.lane_of, self.shapes = [], [], []
        try:
            for i, (rgb, cfg, init, seed) in enumerate(items):
                if isinstance(cfg, dict):
                    cfg = cc.make_config(cfg, seed=seed)
                H, W = rgb.shape[0], rgb.shape[1]
                lane = i % self.lanes
                lib = self.libs[lane]
                h = ctypes.c_void_p()
                rgb = np.ascontiguousarray(rgb, np.uint8)
                _check(lib, lib.cc_init_image(ctypes.byref(cfg), cc._ptr(rgb), H, W,
                                              cc._ptr(init),
                                              cc._stream_handle(self.streams[lane]),
                                              ctypes.byref(h)), "cc_init_image")
                self.ctx.append(h)
                self.lane_of.append(lane)
                self.shapes.append((H, W))
        except Exception:
            self.close()
            raise

    def run(self, iters: int):
        """iters more iterations of every image; returns once all have finished."""
        import torch
        done = 0
        while done < iters:
            n = min(self.chunk, iters - done)
            for i, h in enumerate(self.ctx):
                lib = self.libs[self.lane_of[i]]
                _check(lib, lib.cc_encode_iters(h, n), "cc_encode_iters")
            done += n
        for s in self.streams:
            s.synchronize()
        torch.cuda.synchronize()

    def rd_costs(self, hard: bool = True):
        """(D, R bpp, D + lambda R) of every image (rint latents by default)."""
        out = []
        for i, h in enumerate(self.ctx):
            lib = self.libs[self.lane_of[i]]
            D, R, cost = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            code = lib.cc_rd_cost(h, int(hard), ctypes.byref(D), ctypes.byref(R),
                                  ctypes.byref(cost))
            if code not in (cc.CC_OK, cc.CC_ENONFINITE):
                _check(lib, code, "cc_rd_cost")
            out.append((D.value, R.value, cost.value))
        return out

    def losses(self, i: int, first: int, count: int):
        """D, R and loss of iterations first .. first+count-1 of image i."""
        lib = self.libs[self.lane_of[i]]
        out = np.empty((count, 3), np.float64)
        code = lib.cc_get_losses(self.ctx[i], int(first), int(count), cc._ptr(out))
        if code not in (cc.CC_OK, cc.CC_ENONFINITE):
            _check(lib, code, "cc_get_losses")
        return out

    def set_latents(self, i: int, y_flat):
        """Replace image i's latents (flat latent order, float32, host or device)."""
        lib = self.libs[self.lane_of[i]]
        y = np.ascontiguousarray(y_flat, np.float32) if isinstance(y_flat, np.ndarray) else y_flat
        _check(lib, lib.cc_set_latents(self.ctx[i], cc._ptr(y)), "cc_set_latents")

    def latents(self, i: int):
        """Image i's latents (flat latent order, float32)."""
        lib = self.libs[self.lane_of[i]]
        H, W = self.shapes[i]
        out = np.empty(sum(h * w for h, w in cc.level_shapes(H, W)), np.float32)
        _check(lib, lib.cc_get_latents(self.ctx[i], cc._ptr(out)), "cc_get_latents")
        return out

    def params(self, i: int, n_params: int):
        """Image i's decoder parameters (flat parameter order, float32)."""
        lib = self.libs[self.lane_of[i]]
        out = np.empty(n_params, np.float32)
        _check(lib, lib.cc_get_params(self.ctx[i], cc._ptr(out)), "cc_get_params")
        return out

    def close(self):
        for i, h in enumerate(self.ctx):
            if h:
                self.libs[self.lane_of[i]].cc_free(h)
        self.ctx = []


def autotune(items, lanes_options=(1, 2, 4, 8, 16), chunk_options=(16, 32, 64),
             probe_iters: int = 64, timer=None):
    """Choose (lanes, chunk) for a batch by measurement.

    Each candidate runs the same images on throwaway contexts: one chunk of warm-up (CUDA
    graph capture), then probe_iters timed iterations; the images of the real run are not
    touched.  Lane counts above the number of images are clamped and repeated candidates
    skipped.  Any choice gives bit-identical results, so only the time is compared.
    Returns ((lanes, chunk), {(lanes, chunk): seconds})."""
    import time
    timer = timer or time.perf_counter
    seen, table = set(), {}
    for lanes in lanes_options:
        lanes = max(1, min(lanes, len(items)))
        for chunk in chunk_options:
            if (lanes, chunk) in seen:
                continue
            seen.add((lanes, chunk))
            b = BatchOverfitter(items, lanes=lanes, chunk=chunk)
            try:
                b.run(chunk)
                t0 = timer()
                b.run(probe_iters)
                table[(lanes, chunk)] = timer() - t0
            finally:
                b.close()
    best = min(table, key=lambda k: (table[k], k))
    return best, table
