"""Shared test helpers: option mapping and image comparison."""
import numpy as np

from oracle import drk_oracle as O

TOL_IMAGE = 2e-4      # max abs error per channel, GPU FP32 vs oracle FP64
TOL_GRAD_REL = 1e-3   # per-tensor relative L2 error of gradients


def f32(x):
    return float(np.float32(x))


def oracle_options(opt) -> O.Options:
    """The oracle's options with the float32 values the GPU uses."""
    return O.Options(alpha_min=f32(opt.alpha_min), T_min=f32(opt.T_min), alpha_max=f32(opt.alpha_max),
                     lowpass_sl=f32(opt.lowpass_sl), near=f32(opt.near_plane), bg=tuple(f32(b) for b in opt.bg),
                     order_mode=int(getattr(opt, "order_mode", 0)), cache_len=int(opt.kbuf_capacity),
                     cull_paper=int(getattr(opt, "cull_level", 2) == 3))


def excluded(flags: np.ndarray) -> np.ndarray:
    """Pixels whose result is decided by an FP32-vs-FP64 threshold or depth tie."""
    return (flags & (O.FLAG_T_MIN | O.FLAG_DEPTH_TIE | O.FLAG_STEEP | O.FLAG_CULL)) != 0


def image_error(gpu_rgb: np.ndarray, ref_rgb: np.ndarray, flags: np.ndarray):
    """gpu_rgb, ref_rgb: (3, m) or (3, H, W); returns (max abs err over
    non-excluded pixels, number excluded)."""
    ex = excluded(flags)
    d = np.abs(gpu_rgb.astype(np.float64) - ref_rgb)
    keep = ~ex
    err = float(d[:, keep].max()) if keep.any() else 0.0
    return err, int(ex.sum())


def rel_err(a: np.ndarray, b: np.ndarray) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
