"""ctypes binding of libdrk (include/drk.h).

Argument marshalling only: every step of the rendering path runs in the
library's CUDA kernels.  Torch tensors provide device memory and streams.
If the library is not built, every entry point raises; there is no
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field, fields

import numpy as np
import torch

from . import build as _build

DRK_OK = 0
STATUS = {0: "DRK_OK", 1: "DRK_ERR_INVALID_ARG", 2: "DRK_ERR_OOM", 3: "DRK_ERR_CUDA", 4: "DRK_ERR_CAPACITY",
          5: "DRK_ERR_TIMEOUT", 6: "DRK_ERR_BUSY", 7: "DRK_ERR_NOT_FOUND"}
CULL_NONE, CULL_RECT, CULL_TILE, CULL_PAPER = 0, 1, 2, 3
PARAM_NAMES = ("mu", "quat", "scale", "theta", "eta", "tau", "opacity", "color")


class DrkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)


class drk_params_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("K", C.c_int32), ("sh_degree", C.c_int32)] + [(k, _fp) for k in PARAM_NAMES]


class drk_params_grad_t(C.Structure):
    _fields_ = [(k, _fp) for k in PARAM_NAMES]


class drk_raw_params_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("K", C.c_int32), ("sh_degree", C.c_int32)] + [(k, _fp) for k in PARAM_NAMES]


class drk_adam_t(C.Structure):
    _fields_ = [("lr", C.c_float * 8), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int64)]


class drk_camera_t(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("world_to_cam", C.c_float * 12)]


class drk_options_t(C.Structure):
    _fields_ = [("alpha_min", C.c_float), ("T_min", C.c_float), ("alpha_max", C.c_float),
                ("lowpass_sl", C.c_float), ("near_plane", C.c_float), ("bg", C.c_float * 3),
                ("cull_level", C.c_int32), ("kbuf_capacity", C.c_int32), ("ovf_capacity", C.c_int32),
                ("order_mode", C.c_int32), ("record_chunks", C.c_int32), ("reserved", C.c_int32 * 3)]


class drk_image_t(C.Structure):
    _fields_ = [("rgb", _fp), ("T_final", _fp), ("n_emitted", C.POINTER(C.c_int32)), ("depth", _fp),
                ("normal", _fp)]


class drk_stats_t(C.Structure):
    _fields_ = [("n_visible", C.c_int64), ("n_pairs", C.c_int64), ("n_evals", C.c_int64), ("n_emitted", C.c_int64),
                ("n_extra_passes", C.c_int64), ("n_tiles", C.c_int64), ("n_contrib_evals", C.c_int64),
                ("n_spills", C.c_int64), ("n_replay_evals", C.c_int64), ("n_geo_evals", C.c_int64),
                ("key_bits_depth", C.c_int32),
                ("status", C.c_int32)]


_lib = None


class drk_pipe_peaks_t(C.Structure):
    _fields_ = [("fma_ops", C.c_double), ("ex2_ops", C.c_double), ("rcp_ops", C.c_double), ("cos_ops", C.c_double),
                ("sms", C.c_int32), ("reserved", C.c_int32)]


class drk_serve_timing_t(C.Structure):
    _fields_ = [("arrival_ms", C.c_double), ("start_ms", C.c_double), ("end_ms", C.c_double),
                ("batch_size", C.c_int32), ("status", C.c_int32),
                ("dev_a0_ms", C.c_double), ("dev_a1_ms", C.c_double), ("dev_b1_ms", C.c_double),
                ("dev_r1_ms", C.c_double), ("stream", C.c_int32), ("reserved", C.c_int32)]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libdrk.so (built in-tree by build()).  Raises if it is missing."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libdrk is not built ({path} missing); call __graft_entry__.build()")
        L = C.CDLL(path)
        vp = C.c_void_p
        L.drk_options_default.argtypes = [C.POINTER(drk_options_t)]
        L.drk_options_default.restype = None
        L.drk_last_error.restype = C.c_char_p
        L.drk_version.restype = C.c_char_p
        L.drk_ctx_create.argtypes = [C.c_int, C.POINTER(vp)]
        L.drk_ctx_destroy.argtypes = [vp]
        L.drk_ctx_destroy.restype = None
        L.drk_render.argtypes = [vp, C.POINTER(drk_params_t), C.POINTER(drk_camera_t), C.POINTER(drk_options_t),
                                 C.POINTER(drk_image_t), C.POINTER(vp), vp]
        L.drk_render_backward.argtypes = [vp, C.POINTER(drk_params_t), C.POINTER(drk_camera_t),
                                          C.POINTER(drk_options_t), vp, _fp, C.POINTER(drk_params_grad_t), vp]
        L.drk_state_free.argtypes = [vp]
        L.drk_state_free.restype = None
        L.drk_get_stats.argtypes = [vp, C.POINTER(drk_stats_t)]
        L.drk_sort_pairs.argtypes = [vp, vp, vp, C.c_int64, C.c_int, vp]
        L.drk_sort_pairs_static.argtypes = [vp, vp, C.c_int64, C.c_int, vp]
        L.drk_sort_pairs_static.restype = C.c_int
        L.drk_measure_pipes.argtypes = [C.c_int, C.POINTER(drk_pipe_peaks_t)]
        L.drk_measure_pipes.restype = C.c_int
        L.drk_timing_enable.argtypes = [vp, C.c_int]
        L.drk_stats_enable.argtypes = [vp, C.c_int]
        L.drk_timing_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.drk_launch_count.restype = C.c_int64
        L.drk_serve_create.argtypes = [C.c_int, C.c_size_t, C.c_int, C.POINTER(drk_options_t), C.POINTER(vp)]
        L.drk_serve_add_scene.argtypes = [vp, C.POINTER(drk_params_t), C.POINTER(C.c_int)]
        L.drk_serve_submit.argtypes = [vp, C.c_int, C.POINTER(drk_camera_t), _fp, C.POINTER(C.c_uint64)]
        L.drk_serve_poll.argtypes = [vp, C.c_uint64, C.POINTER(C.c_int), C.POINTER(drk_serve_timing_t)]
        L.drk_serve_wait.argtypes = [vp, C.c_uint64, C.c_double, C.POINTER(drk_serve_timing_t)]
        L.drk_serve_release.argtypes = [vp, C.c_uint64]
        L.drk_serve_inject_alloc_failure.argtypes = [vp, C.c_int]
        L.drk_serve_destroy.argtypes = [vp]
        L.drk_activate.argtypes = [C.POINTER(drk_raw_params_t), C.POINTER(drk_params_grad_t), vp]
        L.drk_activate_backward.argtypes = [C.POINTER(drk_raw_params_t), C.POINTER(drk_params_grad_t),
                                            C.POINTER(drk_params_grad_t), vp]
        L.drk_adam_step.argtypes = [C.POINTER(drk_raw_params_t), C.POINTER(drk_params_grad_t),
                                    C.POINTER(drk_params_grad_t), C.POINTER(drk_params_grad_t),
                                    C.POINTER(drk_adam_t), C.POINTER(drk_params_grad_t), vp]
        L.drk_lr_exponential.restype = C.c_double
        L.drk_lr_exponential.argtypes = [C.c_int64, C.c_double, C.c_double, C.c_int64]
        L.drk_mesh_to_drk.argtypes = [_fp, C.c_int64, _ip, C.c_int64, C.c_int32, _fp, C.POINTER(drk_mesh_options_t),
                                      C.POINTER(drk_params_grad_t), _ip, vp]
        for f in ("drk_activate", "drk_activate_backward", "drk_adam_step", "drk_mesh_to_drk"):
            getattr(L, f).restype = C.c_int
        for f in ("drk_ctx_create", "drk_render", "drk_render_backward", "drk_get_stats", "drk_sort_pairs",
                  "drk_timing_enable", "drk_stats_enable", "drk_timing_read", "drk_serve_create", "drk_serve_add_scene",
                  "drk_serve_submit", "drk_serve_poll", "drk_serve_wait", "drk_serve_release",
                  "drk_serve_inject_alloc_failure", "drk_serve_destroy"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _check(code: int):
    if code != DRK_OK:
        raise DrkError(code, lib().drk_last_error().decode())


# ---------------------------------------------------------------------------
@dataclass
class Options:
    alpha_min: float = float(np.float32(np.exp(-9.0)))
    T_min: float = 1e-4
    alpha_max: float = 0.99
    lowpass_sl: float = 0.70710678
    near_plane: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)
    cull_level: int = CULL_TILE
    kbuf_capacity: int = 16
    ovf_capacity: int = 0
    order_mode: int = 0          # 0 exact order; 1 the paper's cache-sorting (forward only)
    record_chunks: int = 0       # cap on the backward's contributor records (1024 each); 0 = automatic

    def to_c(self) -> drk_options_t:
        o = drk_options_t()
        o.alpha_min, o.T_min, o.alpha_max = self.alpha_min, self.T_min, self.alpha_max
        o.lowpass_sl, o.near_plane = self.lowpass_sl, self.near_plane
        for i in range(3):
            o.bg[i] = float(self.bg[i])
        o.cull_level, o.kbuf_capacity = int(self.cull_level), int(self.kbuf_capacity)
        o.ovf_capacity = int(self.ovf_capacity)
        o.order_mode = int(self.order_mode)
        o.record_chunks = int(self.record_chunks)
        return o


def default_options() -> drk_options_t:
    o = drk_options_t()
    lib().drk_options_default(C.byref(o))
    return o


def camera_c(cam) -> drk_camera_t:
    c = drk_camera_t()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    w = np.asarray(cam.world_to_cam, np.float32).reshape(12)
    for i in range(12):
        c.world_to_cam[i] = float(w[i])
    return c


def _fptr(t: torch.Tensor | None):
    if t is None:
        return None
    assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    return C.cast(C.c_void_p(t.data_ptr()), _fp)


def _stream_ptr(stream) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Context:
    """drk_ctx_t: device scratch pool and counters of the last render."""

    def __init__(self, device: int = 0):
        h = C.c_void_p()
        _check(lib().drk_ctx_create(int(device), C.byref(h)))
        self.handle = h
        self.device = int(device)

    def close(self):
        if self.handle:
            lib().drk_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        s = drk_stats_t()
        _check(lib().drk_get_stats(self.handle, C.byref(s)))
        return {f: getattr(s, f) for f, _ in drk_stats_t._fields_}

    def timing_enable(self, on: bool = True) -> None:
        _check(lib().drk_timing_enable(self.handle, 1 if on else 0))

    def stats_enable(self, on: bool = True) -> None:
        """Collect the forward raster's statistics (default) or not: without
        them n_evals, n_geo_evals, n_contrib_evals, n_emitted and n_spills
        read 0 and the forward runs slightly faster; images are identical."""
        _check(lib().drk_stats_enable(self.handle, 1 if on else 0))

    def timing_read(self) -> dict:
        ms = (C.c_double * 8)()
        cnt = (C.c_int64 * 8)()
        _check(lib().drk_timing_read(self.handle, ms, cnt))
        return {name: (ms[i], cnt[i]) for i, name in enumerate(STAGES)}


STAGES = ("preprocess", "emit", "sort", "raster", "raster_bwd", "preprocess_bwd", "replay_bwd", "record_sort")


def measure_pipes(device: int = 0) -> dict:
    """Measured FP32 FMA and transcendental (ex2, rcp, cos) throughput of one
    GPU, operations per second (drk_measure_pipes)."""
    p = drk_pipe_peaks_t()
    _check(lib().drk_measure_pipes(int(device), C.byref(p)))
    return {f: getattr(p, f) for f, _ in drk_pipe_peaks_t._fields_ if f != "reserved"}


def launch_count() -> int:
    return int(lib().drk_launch_count())


_default_ctx = {}


def default_context(device: int = 0) -> Context:
    if device not in _default_ctx:
        _default_ctx[device] = Context(device)
    return _default_ctx[device]


@dataclass
class DeviceScene:
    """Activated DRK parameters as contiguous float32 CUDA tensors."""
    mu: torch.Tensor
    quat: torch.Tensor
    scale: torch.Tensor
    theta: torch.Tensor
    eta: torch.Tensor
    tau: torch.Tensor
    opacity: torch.Tensor
    color: torch.Tensor
    sh_degree: int = -1

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    @property
    def K(self) -> int:
        return int(self.scale.shape[1])

    @staticmethod
    def from_scene(scene, device="cuda") -> "DeviceScene":
        t = {k: torch.as_tensor(np.ascontiguousarray(getattr(scene, k), np.float32)).to(device).contiguous()
             for k in PARAM_NAMES}
        return DeviceScene(**t, sh_degree=int(scene.sh_degree))

    def tensors(self) -> dict:
        return {k: getattr(self, k) for k in PARAM_NAMES}

    def to_c(self) -> drk_params_t:
        p = drk_params_t()
        p.n, p.K, p.sh_degree = self.n, self.K, int(self.sh_degree)
        for k in PARAM_NAMES:
            setattr(p, k, _fptr(getattr(self, k)))
        return p


class State:
    """drk_state_t of one forward render (needed by the backward)."""

    def __init__(self, handle, ctx: Context):
        self.handle = handle
        self.ctx = ctx   # the context's pool owns the state's memory

    def free(self):
        if self.handle:
            lib().drk_state_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def drk_render(scene: DeviceScene, cam, opt: Options | None = None, ctx: Context | None = None,
               need_state: bool = False, stream=None, out: dict | None = None):
    """Forward render.  Returns (rgb (3, H, W), T_final (H, W), n_emitted (H, W), state|None)."""
    opt = opt or Options()
    ctx = ctx or default_context(scene.mu.device.index or 0)
    H, W = int(cam.height), int(cam.width)
    dev = scene.mu.device
    if out is None:
        out = dict(rgb=torch.empty((3, H, W), device=dev), T=torch.empty((H, W), device=dev),
                   n=torch.empty((H, W), device=dev, dtype=torch.int32))
    img = drk_image_t()
    img.rgb = _fptr(out["rgb"])
    img.T_final = _fptr(out.get("T"))
    img.n_emitted = C.cast(C.c_void_p(out["n"].data_ptr()), C.POINTER(C.c_int32)) if out.get("n") is not None else None
    img.depth = _fptr(out.get("depth"))
    img.normal = _fptr(out.get("normal"))
    p, cc, oc = scene.to_c(), camera_c(cam), opt.to_c()
    h = C.c_void_p()
    _check(lib().drk_render(ctx.handle, C.byref(p), C.byref(cc), C.byref(oc), C.byref(img),
                            C.byref(h) if need_state else None, _stream_ptr(stream)))
    st = State(h, ctx) if need_state else None
    return out["rgb"], out.get("T"), out.get("n"), st


def drk_render_aux(scene: DeviceScene, cam, opt: Options | None = None, ctx: Context | None = None, stream=None):
    """Forward render with the depth and normal images.  Returns (rgb
    (3, H, W), T_final (H, W), depth (H, W), normal (3, H, W)); depth and
    normal are sums weighted by T_i alpha_i (divide by 1 - T_final for the
    mean over the covered part)."""
    H, W = int(cam.height), int(cam.width)
    dev = scene.mu.device
    out = dict(rgb=torch.empty((3, H, W), device=dev), T=torch.empty((H, W), device=dev), n=None,
               depth=torch.empty((H, W), device=dev), normal=torch.empty((3, H, W), device=dev))
    drk_render(scene, cam, opt, ctx=ctx, stream=stream, out=out)
    return out["rgb"], out["T"], out["depth"], out["normal"]


def drk_render_backward(scene: DeviceScene, cam, opt: Options | None, state: State, dL_drgb: torch.Tensor,
                        ctx: Context | None = None, stream=None) -> dict:
    """Reverse mode: gradients of sum(dL_drgb * rgb) for every parameter array."""
    opt = opt or Options()
    ctx = ctx or state.ctx
    grads = {k: torch.empty_like(getattr(scene, k)) for k in PARAM_NAMES}
    g = drk_params_grad_t()
    for k in PARAM_NAMES:
        setattr(g, k, _fptr(grads[k]))
    p, cc, oc = scene.to_c(), camera_c(cam), opt.to_c()
    dL = dL_drgb.contiguous().float()
    _check(lib().drk_render_backward(ctx.handle, C.byref(p), C.byref(cc), C.byref(oc), state.handle, _fptr(dL),
                                     C.byref(g), _stream_ptr(stream)))
    return grads


def drk_sort_pairs(keys: torch.Tensor, vals: torch.Tensor, key_bits: int = 32, ctx: Context | None = None,
                   stream=None) -> None:
    """In-place stable sort of uint32 (stored as int32) keys with their values."""
    assert keys.is_cuda and keys.dtype == torch.int32 and vals.dtype == torch.int32
    assert keys.is_contiguous() and vals.is_contiguous() and keys.numel() == vals.numel()
    ctx = ctx or default_context(keys.device.index or 0)
    _check(lib().drk_sort_pairs(ctx.handle, C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()),
                                keys.numel(), int(key_bits), _stream_ptr(stream)))


def drk_sort_pairs_static(keys: torch.Tensor, vals: torch.Tensor, key_bits: int = 32, stream=None) -> None:
    """drk_sort_pairs for callers that cannot allocate device memory while they
    sort (device memory fixed at start-up, allocation latency not allowed, or
    code inside an allocator's own bookkeeping): the working memory is a
    fixed array inside the library, shared by all calls (order overlapping
    calls yourself).  At most 2^20 pairs.  Runs on the device of `keys`, on
    that device's current stream unless `stream` is given."""
    assert keys.is_cuda and keys.dtype == torch.int32 and vals.dtype == torch.int32
    assert keys.is_contiguous() and vals.is_contiguous() and keys.numel() == vals.numel()
    with torch.cuda.device(keys.device):
        if stream is None:
            stream = torch.cuda.current_stream(keys.device)
        _check(lib().drk_sort_pairs_static(C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()), keys.numel(),
                                           int(key_bits), _stream_ptr(stream)))


class DRKRender(torch.autograd.Function):
    """Differentiable render: (mu, quat, scale, theta, eta, tau, opacity, color) -> rgb (3, H, W).

    Gradients are with respect to the activated parameters."""

    @staticmethod
    def forward(fctx, cam, opt, sh_degree, mu, quat, scale, theta, eta, tau, opacity, color):
        scene = DeviceScene(*(t.detach().contiguous() for t in (mu, quat, scale, theta, eta, tau, opacity, color)),
                            sh_degree=sh_degree)
        rgb, _, _, st = drk_render(scene, cam, opt, need_state=True)
        fctx.scene, fctx.cam, fctx.opt, fctx.state = scene, cam, opt, st
        return rgb

    @staticmethod
    def backward(fctx, dL):
        g = drk_render_backward(fctx.scene, fctx.cam, fctx.opt, fctx.state, dL)
        fctx.state.free()
        return (None, None, None) + tuple(g[k] for k in PARAM_NAMES)


def render_autograd(params: dict, cam, opt: Options | None = None, sh_degree: int = -1) -> torch.Tensor:
    return DRKRender.apply(cam, opt or Options(), sh_degree, *(params[k] for k in PARAM_NAMES))


# ---------------------------------------------------------------------------
# training: activations of the learnable parameters and the fused Adam step

@dataclass
class RawScene:
    """Unconstrained learnable parameters (supplementary "Parametrization"),
    contiguous float32 CUDA tensors with the shapes of DeviceScene.  mu and
    color are used by the renderer as they are."""
    mu: torch.Tensor
    quat: torch.Tensor
    scale: torch.Tensor
    theta: torch.Tensor
    eta: torch.Tensor
    tau: torch.Tensor
    opacity: torch.Tensor
    color: torch.Tensor
    sh_degree: int = -1

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    @property
    def K(self) -> int:
        return int(self.scale.shape[1])

    @staticmethod
    def from_arrays(arrays: dict, sh_degree: int = -1, device="cuda") -> "RawScene":
        t = {k: torch.as_tensor(np.ascontiguousarray(arrays[k], np.float32)).to(device).contiguous()
             for k in PARAM_NAMES}
        return RawScene(**t, sh_degree=int(sh_degree))

    def tensors(self) -> dict:
        return {k: getattr(self, k) for k in PARAM_NAMES}

    def to_c(self) -> drk_raw_params_t:
        p = drk_raw_params_t()
        p.n, p.K, p.sh_degree = self.n, self.K, int(self.sh_degree)
        for k in PARAM_NAMES:
            setattr(p, k, _fptr(getattr(self, k)))
        return p


def _arrays_c(d: dict) -> drk_params_grad_t:
    g = drk_params_grad_t()
    for k in PARAM_NAMES:
        setattr(g, k, _fptr(d.get(k)))
    return g


def activate(raw: RawScene, out: DeviceScene | None = None, stream=None) -> DeviceScene:
    """Activated parameters of raw (drk_activate); the result shares raw's mu
    and color tensors."""
    if out is None:
        out = DeviceScene(raw.mu, *(torch.empty_like(getattr(raw, k)) for k in PARAM_NAMES[1:-1]), raw.color,
                          sh_degree=raw.sh_degree)
    p, o = raw.to_c(), _arrays_c(out.tensors())
    _check(lib().drk_activate(C.byref(p), C.byref(o), _stream_ptr(stream)))
    return out


def activate_backward(raw: RawScene, g_act: dict, stream=None) -> dict:
    """Gradients of the raw parameters from those of the activated ones."""
    g_raw = {k: torch.empty_like(getattr(raw, k)) for k in PARAM_NAMES}
    p, gi, go = raw.to_c(), _arrays_c(g_act), _arrays_c(g_raw)
    _check(lib().drk_activate_backward(C.byref(p), C.byref(gi), C.byref(go), _stream_ptr(stream)))
    return g_raw


# Learning rates (initial, final) decayed log-linearly over max_steps.  The
# supplement fixes the DRK-specific ones (scale, theta, eta, tau: 5e-3 to
# 1e-2 of it at 35K steps); the others follow 3D-GS's published defaults.
LR_SCHEDULE = {"mu": (1.6e-4, 1.6e-6), "quat": (1e-3, 1e-3), "scale": (5e-3, 5e-5), "theta": (5e-3, 5e-5),
               "eta": (5e-3, 5e-5), "tau": (5e-3, 5e-5), "opacity": (5e-2, 5e-2), "color": (2.5e-3, 2.5e-3)}


def lr_exponential(step: int, lr_init: float, lr_final: float, max_steps: int) -> float:
    return float(lib().drk_lr_exponential(int(step), float(lr_init), float(lr_final), int(max_steps)))


def learning_rates(step: int, max_steps: int = 35000, schedule: dict | None = None) -> dict:
    sch = schedule or LR_SCHEDULE
    return {k: lr_exponential(step, *sch[k], max_steps) for k in PARAM_NAMES}


class Adam:
    """Adam on a RawScene from gradients of the activated parameters
    (drk_adam_step: chain rule, update and re-activation in one launch).
    `scene` is the activated DeviceScene the renderer reads; it is updated
    in place by every step."""

    def __init__(self, raw: RawScene, betas=(0.9, 0.999), eps: float = 1e-15, stream=None):
        self.raw = raw
        self.m = {k: torch.zeros_like(getattr(raw, k)) for k in PARAM_NAMES}
        self.v = {k: torch.zeros_like(getattr(raw, k)) for k in PARAM_NAMES}
        self.betas, self.eps, self.t = betas, float(eps), 0
        self.scene = activate(raw, stream=stream)

    def step(self, g_act: dict, lr: dict, stream=None) -> DeviceScene:
        self.t += 1
        hp = drk_adam_t()
        for i, k in enumerate(PARAM_NAMES):
            hp.lr[i] = float(lr[k])
        hp.beta1, hp.beta2, hp.eps, hp.step = float(self.betas[0]), float(self.betas[1]), self.eps, self.t
        p, g = self.raw.to_c(), _arrays_c(g_act)
        m, v, a = _arrays_c(self.m), _arrays_c(self.v), _arrays_c(self.scene.tensors())
        _check(lib().drk_adam_step(C.byref(p), C.byref(g), C.byref(m), C.byref(v), C.byref(hp), C.byref(a),
                                   _stream_ptr(stream)))
        return self.scene


# ---------------------------------------------------------------------------
# mesh to DRK

class drk_mesh_options_t(C.Structure):
    _fields_ = [("K", C.c_int32), ("edge_density", C.c_float), ("tau", C.c_float), ("opacity", C.c_float),
                ("light", C.c_float * 3), ("ambient", C.c_float), ("diffuse", C.c_float)]


@dataclass
class MeshOptions:
    """drk_mesh_options_t (include/drk.h documents every field)."""
    K: int = 4
    edge_density: float = 0.5
    tau: float = 0.95
    opacity: float = 1.0
    light: tuple = (0.3, -0.5, -0.8)
    ambient: float = 0.35
    diffuse: float = 0.65

    def to_c(self) -> drk_mesh_options_t:
        o = drk_mesh_options_t()
        o.K, o.edge_density, o.tau, o.opacity = int(self.K), float(self.edge_density), float(self.tau), \
            float(self.opacity)
        for i in range(3):
            o.light[i] = float(self.light[i])
        o.ambient, o.diffuse = float(self.ambient), float(self.diffuse)
        return o


def mesh_to_drk(verts: torch.Tensor, faces: torch.Tensor, face_color: torch.Tensor | None = None,
                opt: MeshOptions | None = None, stream=None):
    """One DRK per face (drk_mesh_to_drk).  verts (V, 3) float32, faces
    (F, face_size) int32 with -1 padding, face_color (F, 3) or None, all on
    the GPU.  Returns (DeviceScene with sh_degree -1, status (F,) int32)."""
    opt = opt or MeshOptions()
    assert verts.is_cuda and verts.dtype == torch.float32 and verts.is_contiguous()
    assert faces.is_cuda and faces.dtype == torch.int32 and faces.is_contiguous() and faces.dim() == 2
    F, K, dev = int(faces.shape[0]), int(opt.K), verts.device
    sc = DeviceScene(torch.empty((F, 3), device=dev), torch.empty((F, 4), device=dev), torch.empty((F, K), device=dev),
                     torch.empty((F, K), device=dev), torch.empty(F, device=dev), torch.empty(F, device=dev),
                     torch.empty(F, device=dev), torch.empty((F, 3), device=dev), sh_degree=-1)
    status = torch.empty(F, dtype=torch.int32, device=dev)
    o, arr = opt.to_c(), _arrays_c(sc.tensors())
    _check(lib().drk_mesh_to_drk(_fptr(verts), int(verts.shape[0]), C.cast(C.c_void_p(faces.data_ptr()), _ip),
                                 F, int(faces.shape[1]), _fptr(face_color), C.byref(o), C.byref(arr),
                                 C.cast(C.c_void_p(status.data_ptr()), _ip), _stream_ptr(stream)))
    return sc, status


# ---------------------------------------------------------------------------
class Server:
    """drk_serve_t: continuous-batching render server over resident scenes.

    submit() returns a ticket; the image is written into the caller's
    (3, H, W) float32 CUDA tensor, which must stay alive until the ticket is
    done.  wait()/poll() return the ticket's timing record as a dict.
    """

    def __init__(self, device: int = 0, mem_budget: int = 8 << 30, max_batch: int = 16,
                 opt: Options | None = None):
        self.opt = opt or Options()
        oc = self.opt.to_c()
        h = C.c_void_p()
        _check(lib().drk_serve_create(int(device), int(mem_budget), int(max_batch), C.byref(oc), C.byref(h)))
        self.handle = h
        self.device = int(device)

    def close(self):
        if self.handle:
            _check(lib().drk_serve_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_scene(self, scene: DeviceScene) -> int:
        p = scene.to_c()
        sid = C.c_int()
        _check(lib().drk_serve_add_scene(self.handle, C.byref(p), C.byref(sid)))
        return int(sid.value)

    def submit(self, scene_id: int, cam, out_rgb: torch.Tensor) -> int:
        if not (out_rgb.is_cuda and out_rgb.dtype == torch.float32 and out_rgb.is_contiguous()
                and tuple(out_rgb.shape) == (3, int(cam.height), int(cam.width))):
            raise DrkError(1, "out_rgb must be a contiguous float32 CUDA tensor of shape (3, H, W)")
        cc = camera_c(cam)
        tk = C.c_uint64()
        _check(lib().drk_serve_submit(self.handle, int(scene_id), C.byref(cc), _fptr(out_rgb), C.byref(tk)))
        return int(tk.value)

    @staticmethod
    def _timing(t: drk_serve_timing_t) -> dict:
        return {f: getattr(t, f) for f, _ in drk_serve_timing_t._fields_}

    def poll(self, ticket: int):
        done = C.c_int()
        t = drk_serve_timing_t()
        _check(lib().drk_serve_poll(self.handle, C.c_uint64(ticket), C.byref(done), C.byref(t)))
        return bool(done.value), self._timing(t)

    def timeline(self, ticket: int, timeout_ms: float = 60000.0) -> dict:
        """The ticket's timing record once its batch's device timeline is
        filled in (the whole batch has finished; a request can complete
        before its batch does)."""
        import time as _time
        t_end = _time.monotonic() + timeout_ms / 1e3
        while True:
            done, t = self.poll(ticket)
            if done and (t["dev_r1_ms"] > 0.0 or t["status"] != DRK_OK):
                return t
            if _time.monotonic() > t_end:
                raise DrkError(5, "timeline not available")
            _time.sleep(0.001)

    def wait(self, ticket: int, timeout_ms: float = 60000.0) -> dict:
        t = drk_serve_timing_t()
        _check(lib().drk_serve_wait(self.handle, C.c_uint64(ticket), float(timeout_ms), C.byref(t)))
        return self._timing(t)

    def release(self, ticket: int) -> None:
        _check(lib().drk_serve_release(self.handle, C.c_uint64(ticket)))

    def inject_alloc_failure(self, n: int) -> None:
        _check(lib().drk_serve_inject_alloc_failure(self.handle, int(n)))


# ---------------------------------------------------------------------------
# Request-level replicas for serving.

def least_loaded(loads) -> int:
    """Index of the smallest load (the first one on ties)."""
    best = 0
    for i, v in enumerate(loads):
        if v < loads[best]:
            best = i
    return best


class Router:
    """Request-level serving replicas: one Server per entry of `devices` (a
    device may appear more than once), every scene resident on each, every
    request routed to the server with the least outstanding work, counted
    as pixels x primitives of its unfinished requests.  The router
    allocates each request's image on its server's device; image(ticket)
    returns it.  There is no collective and no cross-device traffic: the
    replicas share nothing.

    make_server(device) builds a server (default: Server(device,
    mem_budget, max_batch, opt)); tests pass a stand-in."""

    def __init__(self, devices, mem_budget: int = 8 << 30, max_batch: int = 16, opt: Options | None = None,
                 make_server=None):
        self.devices = [int(d) for d in devices]
        if not self.devices:
            raise DrkError(1, "no devices")
        make = make_server or (lambda d: Server(d, mem_budget=mem_budget, max_batch=max_batch, opt=opt))
        self.servers = [make(d) for d in self.devices]
        self.scene_ids = []          # per scene: its id on every server
        self.scene_n = []            # primitives per scene
        self.load = [0.0] * len(self.servers)
        self.open = {}               # router ticket -> (server index, server ticket, cost, image)
        self.next = 1

    def close(self):
        for s in self.servers:
            s.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_scene(self, scene) -> int:
        """scene: a DeviceScene (copied to each server's device as needed) or
        a host scene with float32 arrays."""
        ids = []
        for srv, dev in zip(self.servers, self.devices):
            if isinstance(scene, DeviceScene):
                ds = scene if scene.mu.device == torch.device("cuda", dev) else DeviceScene(
                    **{k: v.to(torch.device("cuda", dev)) for k, v in scene.tensors().items()},
                    sh_degree=scene.sh_degree)
            else:
                ds = DeviceScene.from_scene(scene, torch.device("cuda", dev))
            ids.append(srv.add_scene(ds))
        self.scene_ids.append(ids)
        self.scene_n.append(int(scene.n if isinstance(scene, DeviceScene) else np.shape(scene.mu)[0]))
        return len(self.scene_ids) - 1

    def _reap(self):
        """Drops finished requests from the loads."""
        for tk, (si, st, cost, _img) in list(self.open.items()):
            if cost > 0.0 and self.servers[si].poll(st)[0]:
                self.load[si] -= cost
                self.open[tk] = (si, st, 0.0, _img)

    def submit(self, scene: int, cam) -> int:
        self._reap()
        si = least_loaded(self.load)
        dev = self.devices[si]
        img = torch.empty((3, int(cam.height), int(cam.width)), dtype=torch.float32, device=torch.device("cuda", dev))
        st = self.servers[si].submit(self.scene_ids[scene][si], cam, img)
        cost = float(cam.width) * float(cam.height) * max(1, self.scene_n[scene])
        self.load[si] += cost
        tk = self.next
        self.next += 1
        self.open[tk] = (si, st, cost, img)
        return tk

    def server_of(self, ticket: int) -> int:
        return self.open[ticket][0]

    def wait(self, ticket: int, timeout_ms: float = 60000.0) -> dict:
        si, st, cost, img = self.open[ticket]
        t = self.servers[si].wait(st, timeout_ms)
        if cost > 0.0:
            self.load[si] -= cost
            self.open[ticket] = (si, st, 0.0, img)
        return t

    def image(self, ticket: int) -> torch.Tensor:
        return self.open[ticket][3]

    def release(self, ticket: int) -> None:
        si, st, cost, _ = self.open.pop(ticket)
        if cost > 0.0:
            self.load[si] -= cost
        self.servers[si].release(st)
