"""Pin of the oracle's float32 error model of alpha_tilde (alpha_fp32_error).

The oracle does not only render: for every pixel it also says how far a
float32 evaluation of the same pixel may land from its FP64 result (the
`tol` budget), and the GPU parity tests hold flagged pixels to that budget.
The budget starts from a per-pair bound on the float32 error of
alpha_tilde.  This test holds that bound against an actual float32
evaluation of Eq. 4 - Eq. 10, written here step by step in numpy float32
(ray, ray-plane intersection, local coordinates, polar angle and sector,
Eq. 6 - Eq. 9, the filter of Eq. 10, the clamp), on 1e5+ random pairs that
include grazing rays (cosine between ray and plane normal down to 1e-3) and
hard edges (tau up to 0.99): every pair's float32 alpha must lie within the
model's bound of the FP64 alpha.
"""
import math

import numpy as np
import pytest

from oracle import drk_oracle as O
from paper_2412_11752_gb300 import synth

f32 = np.float32


def _rot_cols(q):
    """Columns Rx, Ry, Rz of R(q), q = (w, x, y, z) normalised, in float32."""
    q = q / np.sqrt((q * q).sum(axis=1, keepdims=True))
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    one, two = f32(1), f32(2)
    Rx = np.stack([one - two * (y * y + z * z), two * (x * y + w * z), two * (x * z - w * y)], axis=1)
    Ry = np.stack([two * (x * y - w * z), one - two * (x * x + z * z), two * (y * z + w * x)], axis=1)
    Rz = np.stack([two * (x * z + w * y), two * (y * z - w * x), one - two * (x * x + y * y)], axis=1)
    return Rx, Ry, Rz


def _psi(g, tau):
    one, four = f32(1), f32(4)
    lo = g < (one + tau) / four
    mid = g < (f32(3) - tau) / four
    a = (one - tau) / (one + tau) * g
    b = (one + tau) / (one - tau) * g - tau / (one - tau)
    c = (one - tau) / (one + tau) * g + f32(2) * tau / (one + tau)
    return np.where(lo, a, np.where(mid, b, c))


def alpha_float32(scene, cam, opt, idx, pix):
    """alpha_tilde of each (pixel, primitive) pair, every step in float32.
    Returns (valid, alpha, t)."""
    K = scene.scale.shape[1]
    M = np.asarray(cam.world_to_cam, f32).reshape(3, 4)
    Rc, tc = M[:, :3], M[:, 3]
    ocam = -(Rc.T @ tc).astype(f32)
    mu = scene.mu[idx].astype(f32)
    Rx, Ry, Rz = _rot_cols(scene.quat[idx].astype(f32))
    px = pix[:, 0].astype(f32)
    py = pix[:, 1].astype(f32)
    half = f32(0.5)
    dc = np.stack([(px + half - f32(cam.cx)) / f32(cam.fx), (py + half - f32(cam.cy)) / f32(cam.fy),
                   np.ones_like(px)], axis=1)
    d = (dc @ Rc).astype(f32)                       # world ray, camera-space z = 1
    m = (mu - ocam).astype(f32)
    dn = (d * Rz).sum(axis=1)
    dnorm = np.sqrt((d * d).sum(axis=1))
    t = (m * Rz).sum(axis=1) / dn
    valid = (np.abs(dn) >= f32(1e-7) * dnorm) & (t > f32(opt.near))
    p = t[:, None] * d - m                          # Eq. 4 - Eq. 5
    u = (Rx * p).sum(axis=1)
    v = (Ry * p).sum(axis=1)
    th = scene.theta[idx].astype(f32)
    s = scene.scale[idx].astype(f32)
    two_pi = f32(2 * math.pi)
    phi = np.arctan2(v, u)
    rel = np.mod(phi - th[:, 0], two_pi)
    phi = th[:, 0] + rel
    k = (th[:, 1:] < phi[:, None]).sum(axis=1)
    k1 = (k + 1) % K
    rows = np.arange(len(idx))
    th_k = th[rows, k]
    th_k1 = np.where(k + 1 < K, th[rows, np.minimum(k + 1, K - 1)], th[:, 0] + two_pi)
    s_k, s_k1 = s[rows, k], s[rows, k1]
    gap = th_k1 - th_k
    dth = (phi - th_k) * f32(math.pi) / gap        # Eq. 6
    c = np.cos(dth)
    one, two = f32(1), f32(2)
    Q = (one + c) / (two * s_k * s_k) + (one - c) / (two * s_k1 * s_k1)
    e0x, e0y = s_k * np.cos(th_k), s_k * np.sin(th_k)
    e1x, e1y = s_k1 * np.cos(th_k1), s_k1 * np.sin(th_k1)
    det = e0x * e1y - e1x * e0y                     # Eq. 7
    a = (e1y * u - e1x * v) / det
    b = (-e0y * u + e0x * v) / det
    r1 = np.abs(a) + np.abs(b)
    eta = scene.eta[idx].astype(f32)
    E = eta * r1 * r1 + (one - eta) * (u * u + v * v) * Q          # Eq. 8
    g = np.exp(-half * E)
    o = scene.opacity[idx].astype(f32)
    alpha = o * _psi(g, scene.tau[idx].astype(f32))               # Eq. 9
    if opt.lowpass_sl > 0:                                        # Eq. 10
        muc = (mu @ Rc.T + tc).astype(f32)
        infront = muc[:, 2] > f32(opt.near)
        prx = f32(cam.fx) * muc[:, 0] / muc[:, 2] + f32(cam.cx)
        pry = f32(cam.fy) * muc[:, 1] / muc[:, 2] + f32(cam.cy)
        dpx, dpy = px + half - prx, py + half - pry
        cosv = np.abs(dn) / dnorm
        sl = f32(opt.lowpass_sl)
        filt = o * np.exp(-(dpx * dpx + dpy * dpy) / (two * cosv * cosv * sl * sl))
        alpha = np.where(infront & (filt > alpha), filt, alpha)
    alpha = np.minimum(alpha, f32(opt.alpha_max))
    return valid, np.where(valid, alpha, f32(0)), t


def _grazing_scene(n, K, seed):
    """Primitives in front of the camera whose plane normal makes an angle
    with the ray to their centre of cosine logU[1e-3, 1]; tau up to 0.99."""
    rng = np.random.default_rng(seed)
    sc = synth.scene_plain(n, K, seed=seed)
    eye = np.array([0.5, 0.5, -1.5])
    view = sc.mu.astype(np.float64) - eye
    view /= np.linalg.norm(view, axis=1, keepdims=True)
    cosang = np.exp(rng.uniform(np.log(1e-3), 0.0, n))
    rnd = rng.standard_normal((n, 3))
    perp = rnd - (rnd * view).sum(axis=1, keepdims=True) * view
    perp /= np.linalg.norm(perp, axis=1, keepdims=True)
    nrm = cosang[:, None] * view + np.sqrt(1 - cosang ** 2)[:, None] * perp
    tx = np.cross(nrm, rng.standard_normal((n, 3)))
    tx /= np.linalg.norm(tx, axis=1, keepdims=True)
    ty = np.cross(nrm, tx)
    R = np.stack([tx, ty, nrm], axis=2)                         # columns
    from scipy.spatial.transform import Rotation
    xyzw = Rotation.from_matrix(R).as_quat()
    sc.quat = np.ascontiguousarray(xyzw[:, [3, 0, 1, 2]], np.float32)
    hard = rng.random(n) < 0.5
    sc.tau = np.where(hard, rng.uniform(0.9, 0.99, n), rng.uniform(-0.1, 0.99, n)).astype(np.float32)
    sc.opacity = np.where(rng.random(n) < 0.3, rng.uniform(0.9, 0.999, n), sc.opacity).astype(np.float32)
    return sc, R, cosang


def _pairs_near(sc, R, cam, seed, per_prim):
    """Pixels near each primitive: in-plane points within ~3 scales of the
    centre, projected and rounded to a pixel."""
    rng = np.random.default_rng(seed + 1)
    n = sc.mu.shape[0]
    idx = np.repeat(np.arange(n), per_prim)
    rad = rng.uniform(0, 3.0, idx.size) * sc.scale[idx].mean(axis=1)
    ang = rng.uniform(0, 2 * np.pi, idx.size)
    X = sc.mu[idx] + (rad * np.cos(ang))[:, None] * R[idx, :, 0] + (rad * np.sin(ang))[:, None] * R[idx, :, 1]
    M = np.asarray(cam.world_to_cam, np.float64)
    Xc = X @ M[:, :3].T + M[:, 3]
    x = np.floor(cam.fx * Xc[:, 0] / Xc[:, 2] + cam.cx)
    y = np.floor(cam.fy * Xc[:, 1] / Xc[:, 2] + cam.cy)
    ok = (Xc[:, 2] > 0.3) & (x >= 0) & (x < cam.width) & (y >= 0) & (y < cam.height)
    return idx[ok], np.stack([x[ok], y[ok]], axis=1).astype(np.int32)


@pytest.mark.parametrize("K,seed,sl", [(8, 9100, 1 / math.sqrt(2)), (16, 9101, 1 / math.sqrt(2)), (5, 9102, 0.0)])
def test_alpha_error_model_bounds_float32(K, seed, sl):
    cam = synth.camera_front(1920, 1080)
    sc, R, cosang = _grazing_scene(12000, K, seed)
    idx, pix = _pairs_near(sc, R, cam, seed, 12)
    assert idx.size >= 100_000
    opt = O.Options(alpha_min=float(f32(math.exp(-9))), T_min=float(f32(1e-4)), alpha_max=float(f32(0.99)),
                    lowpass_sl=float(f32(sl)), near=float(f32(0.2)))
    ref = O.pairs(sc, cam, opt, idx, pix)
    ok32, a32, t32 = alpha_float32(sc, cam, opt, idx, pix)
    # compare where both take the pair (the near-plane and parallel-ray
    # decisions agree away from their thresholds)
    both = ref["valid"] & ok32 & (np.abs(ref["t"] - opt.near) > 1e-5)
    assert both.mean() > 0.95
    a64, da = ref["alpha"][both], ref["dalpha"][both]
    err = np.abs(a32[both].astype(np.float64) - a64)
    visible = a64 >= opt.alpha_min
    # coverage: grazing rays and hard edges are present among visible pairs
    assert (cosang[idx[both]][visible] < 3e-3).sum() > 50
    assert ((sc.tau[idx[both]] > 0.97) & visible & (a64 > 0.05) & (a64 < 0.9)).sum() > 500
    bound = da + 1e-9
    bad = err > bound
    assert not bad.any(), (f"{bad.sum()} of {err.size} pairs exceed the model: worst err {err[bad].max():.3e} "
                           f"with bound {bound[bad][np.argmax(err[bad])]:.3e}")
    # the model is not vacuous: it is within a few hundred times the error
    # actually made where the error is visible
    big = visible & (err > 1e-6)
    assert np.median(bound[big] / err[big]) < 300
