"""ctypes front end of the FP64 CPU oracle (``drk_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Imported by the test-suite, by the smoke check and
by the benchmark's CPU-baseline leg; never by the product path.  It does not
import the CUDA package and the CUDA package does not import it.

The inputs are the float32 arrays of a scene (any object with the attributes
mu, quat, scale, theta, eta, tau, opacity, color, sh_degree) and of a camera
(width, height, fx, fy, cx, cy, world_to_cam); they are promoted to float64
here.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "drk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libdrk_oracle.so")
_lock = threading.Lock()
_lib = None

FLAG_ALPHA_MIN = 1
FLAG_T_MIN = 2
FLAG_DEPTH_TIE = 4
FLAG_STEEP = 8
FLAG_CULL = 16
FLAG_KINK = 32          # a composited alpha within float32 rounding of a derivative branch point


@dataclass
class Options:
    """Rendering options (the oracle's own copy; the CUDA path has its own)."""
    alpha_min: float = math.exp(-9.0)
    T_min: float = 1e-4
    alpha_max: float = 0.99
    lowpass_sl: float = 1.0 / math.sqrt(2.0)
    near: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)
    order_mode: int = 0          # 0 exact (r_t, index) order; 1 the paper's cache-sorting
    cache_len: int = 8
    cull_paper: int = 0          # 1: the paper's endpoint-polygon tile culling (lossy)


class _Params(C.Structure):
    _fields_ = [("n", C.c_int64), ("K", C.c_int), ("sh_degree", C.c_int)] + [
        (k, C.POINTER(C.c_double)) for k in ("mu", "quat", "scale", "theta", "eta", "tau", "opacity", "color")]


class _Grads(C.Structure):
    _fields_ = [(k, C.POINTER(C.c_double)) for k in
                ("mu", "quat", "scale", "theta", "eta", "tau", "opacity", "color")]


class _Camera(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("w2c", C.c_double * 12)]


class _Options(C.Structure):
    _fields_ = [("alpha_min", C.c_double), ("T_min", C.c_double), ("alpha_max", C.c_double),
                ("lowpass_sl", C.c_double), ("near_plane", C.c_double), ("bg", C.c_double * 3),
                ("order_mode", C.c_int), ("cache_len", C.c_int), ("cull_paper", C.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP, no fast-math)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
                        "-ffp-contract=off", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.ord_psi.restype = C.c_double
        L.ord_psi.argtypes = [C.c_double, C.c_double]
        L.ord_psi_inv.restype = C.c_double
        L.ord_psi_inv.argtypes = [C.c_double, C.c_double]
        L.ord_rotation.argtypes = [dp, dp]
        L.ord_sh_basis.argtypes = [C.c_int, dp, dp]
        L.ord_kernel_uv.restype = C.c_double
        L.ord_kernel_uv.argtypes = [C.c_int, dp, dp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]
        L.ord_l1_norm.restype = C.c_double
        L.ord_l1_norm.argtypes = [C.c_int, dp, dp, C.c_double, C.c_double]
        L.ord_pair.restype = C.c_int
        L.ord_pair.argtypes = [C.POINTER(_Params), C.c_int64, C.POINTER(_Camera), C.POINTER(_Options),
                               C.c_int, C.c_int, dp, dp]
        L.ord_pairs.argtypes = [C.POINTER(_Params), C.POINTER(_Camera), C.POINTER(_Options), C.c_int64,
                                C.POINTER(C.c_int64), C.POINTER(C.c_int32), dp, dp, dp, C.POINTER(C.c_int32)]
        L.ord_color.argtypes = [C.POINTER(_Params), C.c_int64, C.POINTER(_Camera), dp]
        L.ord_render.restype = C.c_int
        L.ord_render.argtypes = [C.POINTER(_Params), C.POINTER(_Camera), C.POINTER(_Options), C.c_int64,
                                 C.POINTER(C.c_int32), dp, dp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), dp]
        L.ord_render_backward.restype = C.c_int
        L.ord_render_backward.argtypes = [C.POINTER(_Params), C.POINTER(_Camera), C.POINTER(_Options), C.c_int64,
                                          C.POINTER(C.c_int32), dp, C.POINTER(_Grads)]
        L.ord_contributors.restype = C.c_int64
        L.ord_contributors.argtypes = [C.POINTER(_Params), C.POINTER(_Camera), C.POINTER(_Options), C.c_int,
                                       C.c_int, C.c_int64, C.POINTER(C.c_int64), dp, dp, C.POINTER(C.c_int64)]
        L.ord_render_aux.restype = C.c_int
        L.ord_render_aux.argtypes = [C.POINTER(_Params), C.POINTER(_Camera), C.POINTER(_Options), C.c_int64,
                                     C.POINTER(C.c_int32), dp, dp]
        L.ord_max_threads.restype = C.c_int
        L.ord_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _Keep:
    """Holds float64 copies alive while a call runs."""

    def __init__(self):
        self.arrs = []

    def f64(self, a):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        self.arrs.append(a)
        return a


def _params(scene, keep: _Keep) -> _Params:
    p = _Params()
    p.n = int(scene.mu.shape[0])
    p.K = int(scene.scale.shape[1])
    p.sh_degree = int(scene.sh_degree)
    for k in ("mu", "quat", "scale", "theta", "eta", "tau", "opacity", "color"):
        setattr(p, k, _dp(keep.f64(getattr(scene, k))))
    return p


def _camera(cam) -> _Camera:
    c = _Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    w = np.asarray(cam.world_to_cam, np.float64).reshape(12)
    for i in range(12):
        c.w2c[i] = float(w[i])
    return c


def _options(opt: Options) -> _Options:
    o = _Options()
    o.alpha_min, o.T_min, o.alpha_max = opt.alpha_min, opt.T_min, opt.alpha_max
    o.lowpass_sl, o.near_plane = opt.lowpass_sl, opt.near
    for i in range(3):
        o.bg[i] = float(opt.bg[i])
    o.order_mode, o.cache_len = int(opt.order_mode), int(opt.cache_len)
    o.cull_paper = int(opt.cull_paper)
    return o


def all_pixels(width: int, height: int) -> np.ndarray:
    ys, xs = np.mgrid[0:height, 0:width]
    return np.ascontiguousarray(np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.int32))


# ---------------------------------------------------------------------------
# scalar pieces (Eq. 6 - Eq. 9)

def psi(g: float, tau: float) -> float:
    return lib().ord_psi(float(g), float(tau))


def psi_inv(y: float, tau: float) -> float:
    return lib().ord_psi_inv(float(y), float(tau))


def rotation(q) -> np.ndarray:
    q = np.ascontiguousarray(np.asarray(q, np.float64))
    R = np.zeros(9)
    lib().ord_rotation(_dp(q), _dp(R))
    return R.reshape(3, 3)


def sh_basis(degree: int, direction) -> np.ndarray:
    d = np.ascontiguousarray(np.asarray(direction, np.float64))
    Y = np.zeros(16)
    lib().ord_sh_basis(int(degree), _dp(d), _dp(Y))
    return Y[: (degree + 1) ** 2]


def kernel_uv(scale, theta, eta, tau, opacity, u, v) -> float:
    s = np.ascontiguousarray(np.asarray(scale, np.float64))
    th = np.ascontiguousarray(np.asarray(theta, np.float64))
    return lib().ord_kernel_uv(len(s), _dp(s), _dp(th), float(eta), float(tau), float(opacity), float(u), float(v))


def l1_norm(scale, theta, u, v) -> float:
    s = np.ascontiguousarray(np.asarray(scale, np.float64))
    th = np.ascontiguousarray(np.asarray(theta, np.float64))
    return lib().ord_l1_norm(len(s), _dp(s), _dp(th), float(u), float(v))


def pair(scene, i: int, cam, opt: Options, px: int, py: int):
    """(valid, alpha_tilde, r_t) of one (pixel, primitive) pair."""
    keep = _Keep()
    P, Cm, O = _params(scene, keep), _camera(cam), _options(opt)
    a, t = C.c_double(), C.c_double()
    ok = lib().ord_pair(C.byref(P), int(i), C.byref(Cm), C.byref(O), int(px), int(py), C.byref(a), C.byref(t))
    return bool(ok), a.value, t.value


def pairs(scene, cam, opt: Options, idx: np.ndarray, pixels: np.ndarray) -> dict:
    """Many (pixel, primitive) pairs at once: valid, alpha_tilde, r_t and the
    float32 error model dalpha of alpha_tilde, each (m,)."""
    keep = _Keep()
    P, Cm, O = _params(scene, keep), _camera(cam), _options(opt)
    ix = np.ascontiguousarray(np.asarray(idx, np.int64))
    pix = np.ascontiguousarray(np.asarray(pixels, np.int32))
    m = ix.shape[0]
    a, t, da = np.zeros(m), np.zeros(m), np.zeros(m)
    ok = np.zeros(m, np.int32)
    lib().ord_pairs(C.byref(P), C.byref(Cm), C.byref(O), m, ix.ctypes.data_as(C.POINTER(C.c_int64)),
                    pix.ctypes.data_as(C.POINTER(C.c_int32)), _dp(a), _dp(t), _dp(da),
                    ok.ctypes.data_as(C.POINTER(C.c_int32)))
    return dict(valid=ok.astype(bool), alpha=a, t=t, dalpha=da)


def color(scene, i: int, cam) -> np.ndarray:
    keep = _Keep()
    P, Cm = _params(scene, keep), _camera(cam)
    out = np.zeros(3)
    lib().ord_color(C.byref(P), int(i), C.byref(Cm), _dp(out))
    return out


# ---------------------------------------------------------------------------
# images

def render_pixels(scene, cam, opt: Options, pixels: np.ndarray):
    """Render listed pixels (int32 (m, 2) of x, y).  Returns dict with
    rgb (m, 3), T (m,), n_contrib (m,), flags (m,), and tol (m,): the
    float32 error budget of each pixel (colour units; ord_render)."""
    keep = _Keep()
    P, Cm, O = _params(scene, keep), _camera(cam), _options(opt)
    pix = np.ascontiguousarray(np.asarray(pixels, np.int32))
    m = pix.shape[0]
    rgb = np.zeros((m, 3))
    T = np.zeros(m)
    nc = np.zeros(m, np.int32)
    fl = np.zeros(m, np.int32)
    tol = np.zeros(m)
    rc = lib().ord_render(C.byref(P), C.byref(Cm), C.byref(O), m, pix.ctypes.data_as(C.POINTER(C.c_int32)),
                          _dp(rgb), _dp(T), nc.ctypes.data_as(C.POINTER(C.c_int32)),
                          fl.ctypes.data_as(C.POINTER(C.c_int32)), _dp(tol))
    if rc != 0:
        raise MemoryError("oracle render: allocation failed")
    return dict(rgb=rgb, T=T, n_contrib=nc, flags=fl, tol=tol)


def render(scene, cam, opt: Options):
    """Full image: rgb (3, H, W), T (H, W), n_contrib (H, W), flags (H, W),
    tol (H, W)."""
    H, W = cam.height, cam.width
    r = render_pixels(scene, cam, opt, all_pixels(W, H))
    return dict(rgb=r["rgb"].T.reshape(3, H, W), T=r["T"].reshape(H, W),
                n_contrib=r["n_contrib"].reshape(H, W), flags=r["flags"].reshape(H, W),
                tol=r["tol"].reshape(H, W))


def render_aux_pixels(scene, cam, opt: Options, pixels: np.ndarray):
    """Depth (m,) and camera-space normal (m, 3) images of listed pixels:
    sums of the compositing weights times r_t and times the plane normal
    oriented towards the camera."""
    keep = _Keep()
    P, Cm, O = _params(scene, keep), _camera(cam), _options(opt)
    pix = np.ascontiguousarray(np.asarray(pixels, np.int32))
    m = pix.shape[0]
    depth, normal = np.zeros(m), np.zeros((m, 3))
    if lib().ord_render_aux(C.byref(P), C.byref(Cm), C.byref(O), m, pix.ctypes.data_as(C.POINTER(C.c_int32)),
                            _dp(depth), _dp(normal)) != 0:
        raise MemoryError("oracle aux render: allocation failed")
    return depth, normal


def render_aux(scene, cam, opt: Options):
    """Full images: depth (H, W), normal (3, H, W)."""
    H, W = cam.height, cam.width
    d, n = render_aux_pixels(scene, cam, opt, all_pixels(W, H))
    return d.reshape(H, W), n.T.reshape(3, H, W)


def render_backward_pixels(scene, cam, opt: Options, pixels: np.ndarray, dL_drgb: np.ndarray) -> dict:
    """Gradient of sum_q dL_drgb[q] . rgb[q] (dL_drgb: (m, 3)) with respect to
    every parameter array of the scene (float64, same shapes)."""
    keep = _Keep()
    P, Cm, O = _params(scene, keep), _camera(cam), _options(opt)
    pix = np.ascontiguousarray(np.asarray(pixels, np.int32))
    g_in = keep.f64(dL_drgb).reshape(-1, 3)
    grads = {k: np.zeros(np.shape(getattr(scene, k)), np.float64)
             for k in ("mu", "quat", "scale", "theta", "eta", "tau", "opacity", "color")}
    G = _Grads()
    for k, v in grads.items():
        setattr(G, k, _dp(v))
    rc = lib().ord_render_backward(C.byref(P), C.byref(Cm), C.byref(O), pix.shape[0],
                                   pix.ctypes.data_as(C.POINTER(C.c_int32)), _dp(g_in), C.byref(G))
    if rc != 0:
        raise MemoryError("oracle backward: allocation failed")
    return grads


def render_backward(scene, cam, opt: Options, dL_drgb: np.ndarray) -> dict:
    """dL_drgb: (3, H, W) image gradient."""
    H, W = cam.height, cam.width
    g = np.asarray(dL_drgb, np.float64).reshape(3, H * W).T
    return render_backward_pixels(scene, cam, opt, all_pixels(W, H), g)


def contributors(scene, cam, opt: Options, px: int, py: int, cap: int = 4096):
    """Sorted contributors of one pixel: (idx, t, alpha, n_composited)."""
    keep = _Keep()
    P, Cm, O = _params(scene, keep), _camera(cam), _options(opt)
    idx = np.zeros(cap, np.int64)
    t = np.zeros(cap)
    a = np.zeros(cap)
    ncomp = C.c_int64()
    cnt = lib().ord_contributors(C.byref(P), C.byref(Cm), C.byref(O), int(px), int(py), cap,
                                 idx.ctypes.data_as(C.POINTER(C.c_int64)), _dp(t), _dp(a), C.byref(ncomp))
    m = min(cnt, cap)
    return idx[:m], t[:m], a[:m], ncomp.value


def max_threads() -> int:
    return lib().ord_max_threads()


def set_threads(n: int) -> None:
    lib().ord_set_threads(int(n))
