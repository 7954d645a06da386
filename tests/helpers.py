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


def undecidable(flags: np.ndarray) -> np.ndarray:
    """Pixels with a discrete float32-undecidable outcome (a stop decision,
    a depth tie or a culling decision within float32 margin)."""
    return (flags & (O.FLAG_T_MIN | O.FLAG_DEPTH_TIE | O.FLAG_CULL)) != 0


def excluded(flags: np.ndarray) -> np.ndarray:
    """Pixels whose result is decided by an FP32-vs-FP64 threshold or depth
    tie, or whose float32 alpha error may exceed half the image tolerance
    (the oracle's flags).  Images check these pixels against their float32
    budget (image_parity); gradient and transmittance checks leave them
    out."""
    return (flags & (O.FLAG_T_MIN | O.FLAG_DEPTH_TIE | O.FLAG_STEEP | O.FLAG_CULL)) != 0


def grad_excluded(flags: np.ndarray) -> np.ndarray:
    """Pixels that carry no dL in gradient tests: the excluded ones, and
    those with a composited alpha within float32 rounding of a point where
    its derivative changes branch (a breakpoint of Psi, Eq. 9; the max of
    Eq. 10; the alpha_max clamp), where the two one-sided gradients differ
    and either is right."""
    return excluded(flags) | ((flags & O.FLAG_KINK) != 0)


def image_parity(gpu_rgb: np.ndarray, ref: dict, max_over_strict: int = 2, what: str = "") -> dict:
    """Every pixel of a GPU image against the oracle.

    gpu_rgb: (3, m) or (3, H, W); ref: the oracle's result for the same
    pixels (rgb of the same shape, or (m, 3) from render_pixels; tol and
    flags per pixel).  Each pixel must lie within TOL_IMAGE plus its float32
    budget `tol` (ord_render: the alpha error model carried through Eq. 1,
    undecidable stops, depth ties and culling decisions; pinned by
    test_oracle_error_model.py); at most `max_over_strict` pixels may need
    more than TOL_IMAGE.  Prints and returns the counts."""
    ref_rgb = np.asarray(ref["rgb"], np.float64)
    if ref_rgb.ndim == 2 and ref_rgb.shape[1] == 3 and gpu_rgb.shape[0] == 3 and ref_rgb.shape[0] != 3:
        ref_rgb = ref_rgb.T
    d = np.abs(gpu_rgb.astype(np.float64) - ref_rgb).max(axis=0).ravel()
    tol = np.asarray(ref["tol"], np.float64).ravel()
    flags = np.asarray(ref["flags"]).ravel()
    lim = TOL_IMAGE + tol
    bad = d > lim
    rep = {"pixels": int(d.size), "max_err": float(d.max()) if d.size else 0.0,
           "over_strict": int((d > TOL_IMAGE).sum()), "undecidable": int(undecidable(flags).sum()),
           "wide_budget": int((tol > 1e-4).sum()),
           "worst_budget_use": float(((d - TOL_IMAGE) / np.maximum(tol, 1e-30))[d > TOL_IMAGE].max())
           if (d > TOL_IMAGE).any() else 0.0}
    print(f"parity {what}: {rep['pixels']} pixels, max err {rep['max_err']:.2e}, {rep['over_strict']} above "
          f"{TOL_IMAGE:g} (all within their float32 budget), {rep['undecidable']} with an undecidable "
          f"stop/tie/culling decision, {rep['wide_budget']} with a budget above 1e-4")
    if bad.any():
        q = int(np.argmax(d - lim))
        raise AssertionError(f"{what}: {int(bad.sum())} pixels beyond 2e-4 + budget; worst pixel #{q}: err {d[q]:.3e}, "
                             f"budget {tol[q]:.3e}, flags {flags[q]}")
    assert rep["over_strict"] <= max_over_strict, f"{what}: {rep['over_strict']} pixels above {TOL_IMAGE:g}"
    return rep


def rel_err(a: np.ndarray, b: np.ndarray) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
