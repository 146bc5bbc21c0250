"""Python binding of the C ABI in include/coolchic.h (argument marshalling only).

Every function here forwards to the CUDA library ``_build/libcoolchic.so``; nothing is
computed in Python.  The library must be built (``python -m paper_2403_11651_gb300.build``);
if it is missing or cannot be loaded, ``load()`` raises -- there is no fallback path.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA); their data
pointers are passed through unchanged.
"""
from __future__ import annotations

import ctypes
import json
import os
from ctypes import POINTER, c_double, c_float, c_int, c_size_t, c_uint64, c_void_p

import numpy as np

from . import build as _build

CC_OK, CC_EINVAL, CC_ENOMEM, CC_ECUDA, CC_ETIMEOUT, CC_ENONFINITE, CC_ESTATE = 0, -1, -2, -3, -4, -5, -6
CC_ESIZE = -7
LEVELS = 7


class CCError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {strerror(code)} ({code})"
        if code == CC_ECUDA:
            msg += f": {_lib().cc_last_cuda_error().decode()}"
        super().__init__(msg)


class cc_config(ctypes.Structure):
    _fields_ = [("levels", c_int), ("arm_ctx", c_int), ("arm_layers", c_int),
                ("up_kernel", c_int), ("up_per_level", c_int), ("syn_hidden", c_int),
                ("syn_res3x3", c_int), ("lam", c_float), ("lr", c_float),
                ("total_iters", c_int), ("ste_frac", c_float), ("seed", c_uint64),
                ("soft_temp", c_float)]


_LIB = None


def _declare(lib):
    P = c_void_p
    sig = {
        "cc_param_count": (c_int, [P, POINTER(c_int)]),
        "cc_latent_count": (c_int, [P, c_int, c_int, POINTER(c_int)]),
        "cc_workspace_size": (c_int, [P, c_int, c_int, POINTER(c_size_t)]),
        "cc_init_image": (c_int, [P, P, c_int, c_int, P, P, POINTER(c_void_p)]),
        "cc_init_image_ws": (c_int, [P, P, c_int, c_int, P, P, P, c_size_t, POINTER(c_void_p)]),
        "cc_set_image": (c_int, [P, P]),
        "cc_encode_iters": (c_int, [P, c_int]),
        "cc_rd_cost": (c_int, [P, c_int, POINTER(c_double), POINTER(c_double), POINTER(c_double)]),
        "cc_decode": (c_int, [P, P]),
        "cc_get_grads": (c_int, [P, P, P]),
        "cc_forward_backward": (c_int, [P, P, c_int, P, POINTER(c_double), POINTER(c_double),
                                        POINTER(c_double)]),
        "cc_get_losses": (c_int, [P, c_int, c_int, P]),
        "cc_get_losses_async": (c_int, [P, c_int, c_int, P]),
        "cc_iteration": (c_int, [P, POINTER(c_int)]),
        "cc_set_latents": (c_int, [P, P]),
        "cc_get_latents": (c_int, [P, P]),
        "cc_set_params": (c_int, [P, P]),
        "cc_get_params": (c_int, [P, P]),
        "cc_noise": (c_int, [P, c_int, P]),
        "cc_profile_phases": (c_int, [P, c_int, P]),
        "cc_graph_kernel_count": (c_int, [P, POINTER(c_int)]),
        "cc_get_state": (c_int, [P, P, POINTER(c_size_t)]),
        "cc_set_state": (c_int, [P, P, c_size_t]),
        "cc_rate_bits_noalloc": (c_int, [P, P, c_int, c_int, P, P, P]),
        "cc_encode_iters_checked": (c_int, [P, c_int, c_int, POINTER(c_int)]),
        "cc_debug_inject": (c_int, [P, c_int, c_int]),
        "cc_free": (None, [P]),
        "cc_strerror": (ctypes.c_char_p, [c_int]),
        "cc_last_cuda_error": (ctypes.c_char_p, []),
        "cc_arm_kernel_ms": (c_int, [P, POINTER(ctypes.c_float)]),
        "cc_write_bitstream": (c_int, [P, P, c_size_t, POINTER(c_size_t)]),
        "cc_bitstream_info": (c_int, [P, c_size_t, P, POINTER(c_int), POINTER(c_int)]),
        "cc_decode_bitstream": (c_int, [P, c_size_t, P, P, P, POINTER(ctypes.c_float)]),
        "cc_warm_param_count": (c_int, [POINTER(c_int)]),
        "cc_warm_create": (c_int, [c_int, c_int, P, P, POINTER(c_void_p)]),
        "cc_warm_predict": (c_int, [P, P, P]),
        "cc_warm_loss_grad": (c_int, [P, P, P, POINTER(c_double), P]),
        "cc_warm_train_step": (c_int, [P, P, P, ctypes.c_float, POINTER(c_double)]),
        "cc_warm_get_params": (c_int, [P, P]),
        "cc_warm_set_params": (c_int, [P, P]),
        "cc_warm_free": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if needed and nvcc is present)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        _LIB = _declare(ctypes.CDLL(path))
    return _LIB


def _lib():
    return load()


def strerror(code: int) -> str:
    return _lib().cc_strerror(code).decode()


def _check(code: int, where: str):
    if code != CC_OK:
        raise CCError(code, where)


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (host or device), or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return c_void_p(a.ctypes.data)
    if isinstance(a, (int, c_void_p)):
        return a if isinstance(a, c_void_p) else c_void_p(a)
    raise TypeError(f"cannot take a data pointer of {type(a)}")


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return c_void_p(stream.cuda_stream)
    return c_void_p(int(stream))


# ----------------------------------------------------------------------- configuration

def make_config(d: dict, seed: int | None = None, lam: float | None = None) -> cc_config:
    """cc_config from a configuration dict (see paper_2403_11651_gb300/configs/*.json)."""
    return cc_config(levels=d.get("levels", LEVELS), arm_ctx=d["arm_ctx"],
                     arm_layers=d["arm_layers"], up_kernel=d["up_kernel"],
                     up_per_level=int(d["up_per_level"]), syn_hidden=d["syn_hidden"],
                     syn_res3x3=d["syn_res3x3"], lam=d["lam"] if lam is None else lam,
                     lr=d["lr"], total_iters=d["total_iters"], ste_frac=d["ste_frac"],
                     seed=(d.get("seed", 0) if seed is None else seed),
                     soft_temp=float(d.get("soft_temp", 0.0)))


def load_config(name: str) -> dict:
    with open(os.path.join(os.path.dirname(__file__), "configs", name + ".json")) as f:
        return json.load(f)


def param_layout(cfg: cc_config):
    """(name, shape) in the flat parameter order of include/coolchic.h."""
    n, c = cfg.arm_ctx, cfg.syn_hidden
    out = []
    for i in range(cfg.arm_layers):
        out += [(f"arm.w{i}", (n, n)), (f"arm.b{i}", (n,))]
    out += [("arm.wout", (2, n)), ("arm.bout", (2,))]
    k = cfg.up_kernel
    if cfg.up_per_level:
        out += [(f"up.f{l}", (k, k)) for l in range(1, LEVELS)]
    else:
        out += [("up.f", (k, k))]
    out += [("syn.wa", (c, LEVELS)), ("syn.ba", (c,)), ("syn.wb", (3, c)), ("syn.bb", (3,))]
    for i in range(cfg.syn_res3x3):
        out += [(f"syn.w3_{i}", (3, 3, 3, 3)), (f"syn.b3_{i}", (3,))]
    return out


def flatten_params(named: dict, cfg: cc_config) -> np.ndarray:
    return np.concatenate([np.asarray(named[k], np.float32).reshape(-1)
                           for k, _ in param_layout(cfg)]).astype(np.float32)


def unflatten_params(flat, cfg: cc_config) -> dict:
    out, k = {}, 0
    for name, shape in param_layout(cfg):
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[k:k + n]).reshape(shape)
        k += n
    return out


def level_shapes(H: int, W: int):
    return [(-(-H // (1 << l)), -(-W // (1 << l))) for l in range(LEVELS)]


def split_latents(flat, H: int, W: int):
    out, k = [], 0
    for h, w in level_shapes(H, W):
        out.append(np.asarray(flat[k:k + h * w]).reshape(h, w))
        k += h * w
    return out


# ----------------------------------------------------------------------- C ABI, same names

def cc_param_count(cfg: cc_config) -> int:
    n = c_int()
    _check(_lib().cc_param_count(ctypes.byref(cfg), ctypes.byref(n)), "cc_param_count")
    return n.value


def cc_latent_count(cfg: cc_config, H: int, W: int) -> int:
    n = c_int()
    _check(_lib().cc_latent_count(ctypes.byref(cfg), H, W, ctypes.byref(n)), "cc_latent_count")
    return n.value


def cc_workspace_size(cfg: cc_config, H: int, W: int) -> int:
    n = c_size_t()
    _check(_lib().cc_workspace_size(ctypes.byref(cfg), H, W, ctypes.byref(n)),
           "cc_workspace_size")
    return n.value


def cc_init_image(cfg: cc_config, rgb_hwc, H: int, W: int, init_params=None, stream=None):
    ctx = c_void_p()
    _check(_lib().cc_init_image(ctypes.byref(cfg), _ptr(rgb_hwc), H, W, _ptr(init_params),
                                _stream_handle(stream), ctypes.byref(ctx)), "cc_init_image")
    return ctx


def cc_init_image_ws(cfg: cc_config, rgb_hwc, H: int, W: int, init_params, stream, workspace,
                     ws_bytes: int):
    ctx = c_void_p()
    _check(_lib().cc_init_image_ws(ctypes.byref(cfg), _ptr(rgb_hwc), H, W, _ptr(init_params),
                                   _stream_handle(stream), _ptr(workspace), ws_bytes,
                                   ctypes.byref(ctx)), "cc_init_image_ws")
    return ctx


def cc_set_image(ctx, rgb_hwc):
    _check(_lib().cc_set_image(ctx, _ptr(rgb_hwc)), "cc_set_image")


def cc_encode_iters(ctx, n_iters: int):
    _check(_lib().cc_encode_iters(ctx, int(n_iters)), "cc_encode_iters")


def cc_rd_cost(ctx, hard_round: bool = True):
    D, R, cost = c_double(), c_double(), c_double()
    code = _lib().cc_rd_cost(ctx, int(bool(hard_round)), ctypes.byref(D), ctypes.byref(R),
                             ctypes.byref(cost))
    if code not in (CC_OK, CC_ENONFINITE):
        _check(code, "cc_rd_cost")
    return D.value, R.value, cost.value


def cc_decode(ctx, H: int, W: int, out=None):
    if out is None:
        out = np.empty((H, W, 3), np.float32)
    _check(_lib().cc_decode(ctx, _ptr(out)), "cc_decode")
    return out


def cc_forward_backward(ctx, n_total: int, noise=None, hard: int = -1, out=None,
                        with_loss: bool = False):
    """(grads, D, R_bpp), or (grads, D, R_bpp, loss) with with_loss."""
    if out is None:
        out = np.empty(n_total, np.float32)
    D, R, L = c_double(), c_double(), c_double()
    code = _lib().cc_forward_backward(ctx, _ptr(noise), int(hard), _ptr(out), ctypes.byref(D),
                                      ctypes.byref(R), ctypes.byref(L))
    if code not in (CC_OK, CC_ENONFINITE):
        _check(code, "cc_forward_backward")
    return (out, D.value, R.value, L.value) if with_loss else (out, D.value, R.value)


def cc_encode_iters_checked(ctx, n_iters: int, check_every: int):
    """(code, iterations kept): CC_OK, or CC_ENONFINITE / CC_ETIMEOUT after a rollback to
    the state before the chunk that went wrong."""
    done = c_int()
    code = _lib().cc_encode_iters_checked(ctx, int(n_iters), int(check_every), ctypes.byref(done))
    if code not in (CC_OK, CC_ENONFINITE, CC_ETIMEOUT):
        _check(code, "cc_encode_iters_checked")
    return code, done.value


CC_FAULT_NAN_GRAD, CC_FAULT_ALLOC, CC_FAULT_ARM_STALL = 1, 2, 3


def cc_debug_inject(ctx, fault: int, at_iteration: int = 0):
    _check(_lib().cc_debug_inject(ctx, int(fault), int(at_iteration)), "cc_debug_inject")


def cc_get_grads(ctx, n_total: int, noise=None, out=None):
    if out is None:
        out = np.empty(n_total, np.float32)
    _check(_lib().cc_get_grads(ctx, _ptr(noise), _ptr(out)), "cc_get_grads")
    return out


def cc_get_losses(ctx, first: int, count: int):
    out = np.empty((count, 3), np.float64)
    code = _lib().cc_get_losses(ctx, int(first), int(count), _ptr(out))
    if code not in (CC_OK, CC_ENONFINITE):
        _check(code, "cc_get_losses")
    return out


def cc_get_losses_async(ctx, first: int, count: int, out):
    """Enqueue the copy of log entries into out (device or pinned host, count x 3 float64);
    read it after the context stream has passed the copy."""
    _check(_lib().cc_get_losses_async(ctx, int(first), int(count), _ptr(out)),
           "cc_get_losses_async")
    return out


def cc_iteration(ctx) -> int:
    t = c_int()
    _check(_lib().cc_iteration(ctx, ctypes.byref(t)), "cc_iteration")
    return t.value


def cc_set_latents(ctx, y_flat):
    _check(_lib().cc_set_latents(ctx, _ptr(y_flat)), "cc_set_latents")


def cc_get_latents(ctx, n_latents: int, out=None):
    if out is None:
        out = np.empty(n_latents, np.float32)
    _check(_lib().cc_get_latents(ctx, _ptr(out)), "cc_get_latents")
    return out


def cc_set_params(ctx, params):
    _check(_lib().cc_set_params(ctx, _ptr(params)), "cc_set_params")


def cc_get_params(ctx, n_params: int, out=None):
    if out is None:
        out = np.empty(n_params, np.float32)
    _check(_lib().cc_get_params(ctx, _ptr(out)), "cc_get_params")
    return out


def cc_noise(ctx, iteration: int, n_latents: int, out=None):
    if out is None:
        out = np.empty(n_latents, np.float32)
    _check(_lib().cc_noise(ctx, int(iteration), _ptr(out)), "cc_noise")
    return out


N_PHASES = 7
PHASES = ["upload+quantize", "arm", "up_fwd", "syn_fwd", "syn_bwd", "up_bwd", "reduce+adam"]


def cc_profile_phases(ctx, reps: int = 10):
    out = np.zeros(N_PHASES, np.float32)
    _check(_lib().cc_profile_phases(ctx, int(reps), _ptr(out)), "cc_profile_phases")
    return out


def cc_arm_kernel_ms(ctx) -> float:
    """Milliseconds of the ARM kernel in the most recent pass that ran it on its own stream."""
    ms = ctypes.c_float()
    _check(_lib().cc_arm_kernel_ms(ctx, ctypes.byref(ms)), "cc_arm_kernel_ms")
    return float(ms.value)


def cc_graph_kernel_count(ctx) -> int:
    n = c_int()
    _check(_lib().cc_graph_kernel_count(ctx, ctypes.byref(n)), "cc_graph_kernel_count")
    return n.value


def cc_get_state(ctx) -> bytes:
    n = c_size_t()
    _check(_lib().cc_get_state(ctx, None, ctypes.byref(n)), "cc_get_state")
    buf = ctypes.create_string_buffer(n.value)
    _check(_lib().cc_get_state(ctx, buf, ctypes.byref(n)), "cc_get_state")
    return buf.raw[:n.value]


def cc_set_state(ctx, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(_lib().cc_set_state(ctx, buf, len(blob)), "cc_set_state")


def cc_rate_bits_noalloc(cfg: cc_config, yhat_flat, H: int, W: int, params, stream=None,
                         out=None):
    """Total rate (bits) of a quantised pyramid, computed without allocating device memory.
    With out (a one-element float64 tensor, host or device) the total is written there and
    out is returned; otherwise it is returned as a float."""
    if out is None:
        v = c_double()
        _check(_lib().cc_rate_bits_noalloc(ctypes.byref(cfg), _ptr(yhat_flat), H, W,
                                           _ptr(params), _stream_handle(stream),
                                           ctypes.byref(v)), "cc_rate_bits_noalloc")
        return v.value
    n_out = out.size if isinstance(out, np.ndarray) else out.numel()
    if str(out.dtype) not in ("torch.float64", "float64") or n_out < 1:
        raise ValueError("cc_rate_bits_noalloc: out must hold one float64")
    _check(_lib().cc_rate_bits_noalloc(ctypes.byref(cfg), _ptr(yhat_flat), H, W, _ptr(params),
                                       _stream_handle(stream), _ptr(out)),
           "cc_rate_bits_noalloc")
    return out


def bitstream_bound(cfg: cc_config, H: int, W: int) -> int:
    """Bytes that always hold a bitstream of this configuration and size: the header, the
    parameters, 5 LEB128 bytes per row and the encoder's per-row reservation 8 w + 16."""
    shapes = level_shapes(H, W)
    return (20 + 4 * cc_param_count(cfg) + 5 * sum(h for h, _ in shapes)
            + sum(h * (8 * w + 16) for h, w in shapes))


def cc_write_bitstream(ctx, cfg: cc_config = None, H: int = 0, W: int = 0) -> bytes:
    """Range-coded bitstream of rint(y) and the decoder parameters of the context.  With
    (cfg, H, W) the output buffer is sized from bitstream_bound and the library runs once;
    without, a first call asks for the size."""
    n = c_size_t()
    if cfg is None:
        _check(_lib().cc_write_bitstream(ctx, None, 0, ctypes.byref(n)), "cc_write_bitstream")
        cap = n.value
    else:
        cap = bitstream_bound(cfg, H, W)
    buf = np.empty(max(1, cap), np.uint8)          # not zero-filled
    _check(_lib().cc_write_bitstream(ctx, _ptr(buf), cap, ctypes.byref(n)), "cc_write_bitstream")
    return buf[:n.value].tobytes()


def cc_bitstream_info(bs: bytes):
    """(cc_config with the architecture fields, H, W) of a bitstream."""
    cfg, H, W = cc_config(), c_int(), c_int()
    buf = ctypes.create_string_buffer(bs, len(bs))
    _check(_lib().cc_bitstream_info(buf, len(bs), ctypes.byref(cfg), ctypes.byref(H),
                                    ctypes.byref(W)), "cc_bitstream_info")
    return cfg, H.value, W.value


def cc_decode_bitstream(bs: bytes, rgb_out=None, latents_out=None, stream=None, want_rgb=True,
                        want_latents=True):
    """Decode a bitstream: (image H x W x 3 float32 or None, int32 latents or None, ms of
    the latent decoding)."""
    cfg, H, W = cc_bitstream_info(bs)
    if want_rgb and rgb_out is None:
        rgb_out = np.empty((H, W, 3), np.float32)
    if want_latents and latents_out is None:
        latents_out = np.empty(cc_latent_count(cfg, H, W), np.int32)
    ms = ctypes.c_float()
    buf = ctypes.create_string_buffer(bs, len(bs))
    _check(_lib().cc_decode_bitstream(buf, len(bs), _stream_handle(stream),
                                      _ptr(rgb_out) if want_rgb else None,
                                      _ptr(latents_out) if want_latents else None,
                                      ctypes.byref(ms)), "cc_decode_bitstream")
    return (rgb_out if want_rgb else None), (latents_out if want_latents else None), ms.value


WARM_LAYOUT = ([("c1.w", (32, 3, 3, 3)), ("c1.b", (32,))]
               + [x for i in (2, 3, 4) for x in ((f"c{i}.w", (32, 32, 3, 3)), (f"c{i}.b", (32,)))]
               + [x for i in (1, 2, 3, 4) for x in ((f"h{i}.w", (1, 32, 1, 1)), (f"h{i}.b", (1,)))]
               + [("h0.w", (1, 3, 3, 3)), ("h0.b", (1,))])


def cc_warm_param_count() -> int:
    n = c_int()
    _check(_lib().cc_warm_param_count(ctypes.byref(n)), "cc_warm_param_count")
    return n.value


def cc_warm_create(H: int, W: int, params, stream=None):
    w = c_void_p()
    _check(_lib().cc_warm_create(H, W, _ptr(params), _stream_handle(stream), ctypes.byref(w)),
           "cc_warm_create")
    return w


def cc_warm_predict(w, rgb_hwc, n_latents: int, out=None):
    if out is None:
        out = np.empty(n_latents, np.float32)
    _check(_lib().cc_warm_predict(w, _ptr(rgb_hwc), _ptr(out)), "cc_warm_predict")
    return out


def cc_warm_loss_grad(w, rgb_hwc, target_latents, grads_out=None) -> float:
    loss = c_double()
    _check(_lib().cc_warm_loss_grad(w, _ptr(rgb_hwc), _ptr(target_latents), ctypes.byref(loss),
                                    _ptr(grads_out)), "cc_warm_loss_grad")
    return loss.value


def cc_warm_train_step(w, rgb_hwc, target_latents, lr: float, with_loss: bool = True,
                       loss_out=None):
    """One training step.  Returns the loss (synchronising); with loss_out (a device
    float64 tensor, or its element) the loss is written there on the stream and None is
    returned; with with_loss=False nothing is written (queued only)."""
    if loss_out is not None:
        _check(_lib().cc_warm_train_step(w, _ptr(rgb_hwc), _ptr(target_latents), float(lr),
                                         ctypes.cast(ctypes.c_void_p(loss_out.data_ptr()),
                                                     POINTER(c_double))),
               "cc_warm_train_step")
        return None
    loss = c_double()
    _check(_lib().cc_warm_train_step(w, _ptr(rgb_hwc), _ptr(target_latents), float(lr),
                                     ctypes.byref(loss) if with_loss else None),
           "cc_warm_train_step")
    return loss.value if with_loss else None


def cc_warm_get_params(w, out=None):
    if out is None:
        out = np.empty(cc_warm_param_count(), np.float32)
    _check(_lib().cc_warm_get_params(w, _ptr(out)), "cc_warm_get_params")
    return out


def cc_warm_set_params(w, params):
    _check(_lib().cc_warm_set_params(w, _ptr(params)), "cc_warm_set_params")


def cc_warm_free(w):
    if w:
        _lib().cc_warm_free(w)


def cc_free(ctx):
    if ctx:
        _lib().cc_free(ctx)


def cc_strerror(code: int) -> str:
    return strerror(code)


EXPORTED = ["cc_param_count", "cc_latent_count", "cc_workspace_size", "cc_init_image",
            "cc_init_image_ws", "cc_set_image", "cc_encode_iters", "cc_rd_cost", "cc_decode",
            "cc_get_grads", "cc_forward_backward", "cc_get_losses", "cc_get_losses_async",
            "cc_iteration", "cc_noise",
            "cc_set_latents", "cc_get_latents", "cc_set_params", "cc_get_params",
            "cc_profile_phases", "cc_graph_kernel_count", "cc_arm_kernel_ms", "cc_rate_bits_noalloc",
            "cc_get_state", "cc_set_state", "cc_write_bitstream", "cc_bitstream_info",
            "cc_decode_bitstream", "cc_warm_param_count", "cc_warm_create", "cc_warm_predict",
            "cc_warm_loss_grad", "cc_warm_train_step", "cc_warm_get_params",
            "cc_warm_set_params", "cc_warm_free", "cc_free", "cc_strerror",
            "cc_last_cuda_error", "cc_encode_iters_checked", "cc_debug_inject"]
