"""FP64 oracle of the learnable-parameter activations (supplementary
"Parametrization") and of the optimiser step used to fit them ("Model
Training": Adam as in 3D-GS, exponential learning-rate decay).

TEST INFRASTRUCTURE ONLY.  Imported by the test-suite; never by the product
path.  Plain numpy in float64; it shares no code with the CUDA library.

Readings where the paper is silent:
  T1  theta: w_j = sigmoid(x_j) + 1/(K-2) for j = 0..K-1 (the residual of the
      supplement), theta_0 = 0 and theta_k = 2 pi (w_0 + ... + w_{k-1}) / S
      with S = w_0 + ... + w_{K-1}, so the cumulative sum ends at 2 pi and the
      cyclic gap after theta_k is 2 pi w_k / S.  Every gap is below pi: the
      bound is reached only when one sigmoid is 1 and all others 0.  Because
      float32 sigmoids do saturate, sigmoid(x_j) is capped at c = 1 - 1e-3,
      which keeps every gap at most pi (1 - 1e-3 / (2 - 1e-3 + 2 / (K - 2))),
      below pi (1 - 2.4e-4) for every K >= 3 (gradient 0 above the cap).
  T2  tau = -0.1 + 1.09 sigmoid(x): the supplement's bounds (-0.1, 0.99)
      reached by a sigmoid and a linear remap.
  T3  q = x / |x| (x = 0 gives the identity rotation (1, 0, 0, 0), gradient 0);
      mu and colour (RGB or SH coefficients) are used as they are.
  T4  Adam (Kingma and Ba) with bias correction, the update
      p -= lr / (1 - b1^t) * m / (sqrt(v) / sqrt(1 - b2^t) + eps), t >= 1,
      one learning rate per parameter array.
  T5  learning-rate decay from lr_init to lr_final over max_steps, log-linear
      (lr_init^(1-r) lr_final^r, r = min(step / max_steps, 1)); the
      supplement's DRK-specific rate is 5e-3 decayed to 1e-2 of it at 35K
      steps.
"""
from __future__ import annotations

import math

import numpy as np

ACTIVATED = ("quat", "scale", "theta", "eta", "tau", "opacity")
ALL = ("mu", "quat", "scale", "theta", "eta", "tau", "opacity", "color")
SIG_CAP = 1.0 - 1e-3
TAU_LO, TAU_SPAN = -0.1, 1.09


def sigmoid(x):
    x = np.asarray(x, np.float64)
    with np.errstate(over="ignore"):          # exp(-x) = inf gives 0 exactly
        return 1.0 / (1.0 + np.exp(-x))


def dsigmoid(x):
    """sigmoid'(x) = sigmoid(x) sigmoid(-x), accurate where s (1 - s) cancels."""
    return sigmoid(x) * sigmoid(-np.asarray(x, np.float64))


def theta_from_raw(x: np.ndarray) -> np.ndarray:
    """(n, K) raw angles -> (n, K) polar angles, reading T1."""
    x = np.asarray(x, np.float64)
    K = x.shape[-1]
    w = np.minimum(sigmoid(x), SIG_CAP) + 1.0 / (K - 2)
    S = w.sum(axis=-1, keepdims=True)
    before = np.cumsum(w, axis=-1) - w            # w_0 + ... + w_{k-1}
    return 2.0 * math.pi * before / S


def activate(raw: dict) -> dict:
    """Activated parameters from raw ones (dict of float arrays with the
    shapes of a scene's parameters)."""
    out = {"mu": np.asarray(raw["mu"], np.float64).copy(), "color": np.asarray(raw["color"], np.float64).copy()}
    x = np.asarray(raw["quat"], np.float64)
    nrm = np.linalg.norm(x, axis=-1, keepdims=True)
    q = np.where(nrm > 0, x / np.where(nrm > 0, nrm, 1.0), np.array([1.0, 0.0, 0.0, 0.0]))
    out["quat"] = q
    out["scale"] = np.exp(np.asarray(raw["scale"], np.float64))
    out["theta"] = theta_from_raw(raw["theta"])
    out["eta"] = sigmoid(raw["eta"])
    out["tau"] = TAU_LO + TAU_SPAN * sigmoid(raw["tau"])
    out["opacity"] = sigmoid(raw["opacity"])
    return out


def activate_backward(raw: dict, g: dict) -> dict:
    """Gradient with respect to the raw parameters of sum(g[k] * activated[k])."""
    out = {"mu": np.asarray(g["mu"], np.float64).copy(), "color": np.asarray(g["color"], np.float64).copy()}
    x = np.asarray(raw["quat"], np.float64)
    nrm = np.linalg.norm(x, axis=-1, keepdims=True)
    safe = np.where(nrm > 0, nrm, 1.0)
    q = x / safe
    gq = np.asarray(g["quat"], np.float64)
    out["quat"] = np.where(nrm > 0, (gq - q * np.sum(q * gq, axis=-1, keepdims=True)) / safe, 0.0)
    out["scale"] = np.asarray(g["scale"], np.float64) * np.exp(np.asarray(raw["scale"], np.float64))
    # theta_k = 2 pi C_k / S:  d theta_k / d w_j = 2 pi ([j < k] / S - C_k / S^2)
    xt = np.asarray(raw["theta"], np.float64)
    K = xt.shape[-1]
    sg = sigmoid(xt)
    w = np.minimum(sg, SIG_CAP) + 1.0 / (K - 2)
    S = w.sum(axis=-1, keepdims=True)
    Ck = np.cumsum(w, axis=-1) - w
    gt = np.asarray(g["theta"], np.float64)
    after = np.cumsum(gt[..., ::-1], axis=-1)[..., ::-1] - gt   # sum over k > j of g_k
    gw = 2.0 * math.pi * (after / S - np.sum(gt * Ck, axis=-1, keepdims=True) / S ** 2)
    out["theta"] = gw * np.where(sg < SIG_CAP, dsigmoid(xt), 0.0)
    for k, scale in (("eta", 1.0), ("tau", TAU_SPAN), ("opacity", 1.0)):
        out[k] = np.asarray(g[k], np.float64) * scale * dsigmoid(raw[k])
    return out


def lr_exponential(step: int, lr_init: float, lr_final: float, max_steps: int) -> float:
    """Reading T5."""
    r = min(max(step / max_steps, 0.0), 1.0) if max_steps > 0 else 1.0
    return math.exp((1.0 - r) * math.log(lr_init) + r * math.log(lr_final))


def adam(p, g, m, v, lr: float, step: int, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15):
    """One Adam step (reading T4); returns new (p, m, v)."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    denom = np.sqrt(v) / math.sqrt(1.0 - beta2 ** step) + eps
    return p - lr / (1.0 - beta1 ** step) * m / denom, m, v


def train_step(raw: dict, g_act: dict, m: dict, v: dict, lr: dict, step: int, beta1: float = 0.9,
               beta2: float = 0.999, eps: float = 1e-15):
    """Raw gradients from gradients of the activated parameters, one Adam step
    per array, and the activation of the new raw parameters.  Returns
    (raw, m, v, activated)."""
    g_raw = activate_backward(raw, g_act)
    nr, nm, nv = {}, {}, {}
    for k in ALL:
        nr[k], nm[k], nv[k] = adam(raw[k], g_raw[k], m[k], v[k], lr[k], step, beta1, beta2, eps)
    return nr, nm, nv, activate(nr)
