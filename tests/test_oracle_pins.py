"""Pins of the FP64 oracle against what the paper and mathematics fix.

Every check here uses a route other than the oracle's own formula: a special
case that reduces to another closed form (Eq. 3 from Eq. 6), a library
routine for a convention (scipy rotations and spherical harmonics), an
invariance the method must have, or central finite differences for the
derivative.  No GPU.
"""
import math

import numpy as np
import pytest

from oracle import drk_oracle as O
from paper_2412_11752_gb300 import synth

TWO_PI = 2 * math.pi


# ---------------------------------------------------------------------------
# Eq. 9: sharpening

@pytest.mark.parametrize("tau", [-0.9, -0.1, 0.0, 0.3, 0.7, 0.99])
def test_psi_endpoints_continuity_monotone(tau):
    assert O.psi(0.0, tau) == pytest.approx(0.0, abs=1e-15)
    assert O.psi(1.0, tau) == pytest.approx(1.0, abs=1e-12)
    # both breakpoints: left and right limits agree, with the values the
    # paper's figure implies ((1 - tau)/4 and (3 + tau)/4)
    b1, b2 = (1 + tau) / 4, (3 - tau) / 4
    eps = 1e-12
    assert O.psi(b1 - eps, tau) == pytest.approx(O.psi(b1, tau), abs=1e-9)
    assert O.psi(b2 - eps, tau) == pytest.approx(O.psi(b2, tau), abs=1e-9)
    assert O.psi(b1, tau) == pytest.approx((1 - tau) / 4, abs=1e-12)
    assert O.psi(b2, tau) == pytest.approx((3 + tau) / 4, abs=1e-12)
    g = np.linspace(0, 1, 2001)
    y = np.array([O.psi(x, tau) for x in g])
    assert np.all(np.diff(y) > 0)
    # inverse both ways
    for x in g[::50]:
        assert O.psi_inv(O.psi(x, tau), tau) == pytest.approx(x, abs=1e-12)
        assert O.psi(O.psi_inv(x, tau), tau) == pytest.approx(x, abs=1e-12)


def test_psi_identity_at_zero_sharpness():
    for g in np.linspace(0, 1, 101):
        assert O.psi(g, 0.0) == pytest.approx(g, abs=1e-15)


def test_psi_sharpens_towards_0_and_1():
    # tau > 0 pushes low densities down and high densities up (Sec. 4.3)
    for tau in (0.2, 0.6, 0.95):
        assert O.psi(0.1, tau) < 0.1
        assert O.psi(0.9, tau) > 0.9


# ---------------------------------------------------------------------------
# conventions pinned to library routines

def test_rotation_matches_scipy():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(0)
    for _ in range(50):
        q = rng.standard_normal(4) * rng.uniform(0.2, 3.0)
        R = O.rotation(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(R, ref, atol=1e-13)


def test_identity_quaternion_primitive_lies_in_xy_plane():
    R = O.rotation([1, 0, 0, 0])
    np.testing.assert_allclose(R[:, 2], [0, 0, 1], atol=0)   # normal R_z = world z


def _real_sh_scipy(l, m, d):
    from scipy.special import sph_harm_y
    x, y, z = d
    polar = math.acos(max(-1.0, min(1.0, z)))
    azim = math.atan2(y, x)
    if m == 0:
        return sph_harm_y(l, 0, polar, azim).real
    Y = sph_harm_y(l, abs(m), polar, azim)
    return math.sqrt(2) * (Y.imag if m < 0 else Y.real)


def test_sh_basis_matches_scipy_real_harmonics():
    rng = np.random.default_rng(1)
    for _ in range(40):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        Y = O.sh_basis(3, d)
        ref = [_real_sh_scipy(l, m, d) for l in range(4) for m in range(-l, l + 1)]
        np.testing.assert_allclose(Y, ref, atol=1e-12)


# ---------------------------------------------------------------------------
# Eq. 6 - Eq. 8: kernel special cases

def _rand_uv(rng, n, r=0.3):
    return rng.uniform(-r, r, size=(n, 2))


@pytest.mark.parametrize("su,sv", [(0.05, 0.05), (0.03, 0.08), (0.1, 0.02)])
def test_gaussian_special_case_eq3(su, sv):
    # K = 4, theta_k = k pi / 2, s0 = s2 = su, s1 = s3 = sv, eta = 0, tau = 0
    # reduces Eq. 6 to the 2D Gaussian of Eq. 3 (Sec. 4.1).
    th = [0, math.pi / 2, math.pi, 3 * math.pi / 2]
    s = [su, sv, su, sv]
    o = 0.8
    rng = np.random.default_rng(2)
    for u, v in _rand_uv(rng, 300, 3 * max(su, sv)):
        ref = o * math.exp(-0.5 * (u * u / su ** 2 + v * v / sv ** 2))
        assert O.kernel_uv(s, th, 0.0, 0.0, o, u, v) == pytest.approx(ref, rel=1e-12, abs=1e-300)


def test_isotropic_gaussian_any_angles():
    # equal scales, pure L2, no sharpening: o exp(-r^2 / (2 s^2)) for any angles
    rng = np.random.default_rng(3)
    for K in (3, 5, 8, 16):
        th = synth._angles(rng, 1, K)[0]
        s = np.full(K, 0.04)
        for u, v in _rand_uv(rng, 100, 0.15):
            ref = 0.7 * math.exp(-(u * u + v * v) / (2 * 0.04 ** 2))
            assert O.kernel_uv(s, th, 0.0, 0.0, 0.7, u, v) == pytest.approx(ref, rel=1e-12, abs=1e-300)


def test_l1_diamond_right_angles():
    # eta = 1 with K = 4 right angles: r1 = |u|/su + |v|/sv (the L1 ball of Sec. 4.2)
    th = [0, math.pi / 2, math.pi, 3 * math.pi / 2]
    su, sv = 0.05, 0.09
    s = [su, sv, su, sv]
    rng = np.random.default_rng(4)
    for u, v in _rand_uv(rng, 300, 0.2):
        r1 = abs(u) / su + abs(v) / sv
        assert O.l1_norm(s, th, u, v) == pytest.approx(r1, rel=1e-12)
        assert O.kernel_uv(s, th, 1.0, 0.0, 0.9, u, v) == pytest.approx(0.9 * math.exp(-0.5 * r1 * r1),
                                                                        rel=1e-11, abs=1e-300)


def test_l1_barycentric_in_sector():
    # a point a e_k + b e_{k+1} with a, b >= 0 has r1 = a + b (Eq. 7)
    rng = np.random.default_rng(5)
    for K in (3, 4, 8, 16):
        th = synth._angles(rng, 1, K)[0]
        s = np.exp(rng.normal(-3, 0.5, K))
        for _ in range(50):
            k = int(rng.integers(0, K))
            k1 = (k + 1) % K
            a, b = rng.uniform(0, 2, 2)
            e0 = s[k] * np.array([math.cos(th[k]), math.sin(th[k])])
            e1 = s[k1] * np.array([math.cos(th[k1]), math.sin(th[k1])])
            p = a * e0 + b * e1
            assert O.l1_norm(s, th, p[0], p[1]) == pytest.approx(a + b, rel=1e-10)


def _roll(th, s, m):
    K = len(th)
    th2 = np.array([th[(j + m) % K] + (TWO_PI if j + m >= K else 0.0) for j in range(K)])
    s2 = np.array([s[(j + m) % K] for j in range(K)])
    return th2, s2


def test_cyclic_relabelling_invariance():
    rng = np.random.default_rng(6)
    for K in (3, 5, 8, 16):
        th = synth._angles(rng, 1, K)[0]
        s = np.exp(rng.normal(-3, 0.5, K))
        eta, tau, o = 0.4, 0.5, 0.7
        for m in range(1, K):
            th2, s2 = _roll(th, s, m)
            for u, v in _rand_uv(rng, 20, 0.15):
                a = O.kernel_uv(s, th, eta, tau, o, u, v)
                b = O.kernel_uv(s2, th2, eta, tau, o, u, v)
                assert b == pytest.approx(a, rel=1e-9, abs=1e-300)


def test_in_plane_rotation_invariance():
    # rotating the angles by phi and the point by phi leaves alpha unchanged
    rng = np.random.default_rng(7)
    th = synth._angles(rng, 1, 8)[0]
    s = np.exp(rng.normal(-3, 0.5, 8))
    for phi in (0.3, 1.7, -2.2):
        c, sn = math.cos(phi), math.sin(phi)
        for u, v in _rand_uv(rng, 40, 0.15):
            a = O.kernel_uv(s, th, 0.3, 0.2, 0.9, u, v)
            b = O.kernel_uv(s, th + phi, 0.3, 0.2, 0.9, c * u - sn * v, sn * u + c * v)
            assert b == pytest.approx(a, rel=1e-9, abs=1e-300)


def test_kernel_continuous_across_sector_boundaries():
    rng = np.random.default_rng(8)
    th = synth._angles(rng, 1, 8)[0]
    s = np.exp(rng.normal(-3, 0.5, 8))
    for j in range(8):
        for r in (0.02, 0.06):
            vals = [O.kernel_uv(s, th, 0.5, 0.3, 0.9, r * math.cos(th[j] + e), r * math.sin(th[j] + e))
                    for e in (-1e-9, 0.0, 1e-9)]
            assert max(vals) - min(vals) < 1e-6


def test_sector_wrap_uses_first_scale():
    # points just below theta_0 belong to the wrap sector (theta_{K-1}, theta_0 + 2 pi]
    th = np.array([0.5, 2.0, 4.0])
    s = np.array([0.03, 0.05, 0.07])
    # on the ray theta_0 exactly the L2 radius is s_0
    r = 0.03
    a = O.kernel_uv(s, th, 0.0, 0.0, 1.0, r * math.cos(0.5 - 1e-12), r * math.sin(0.5 - 1e-12))
    assert a == pytest.approx(math.exp(-0.5), rel=1e-6)


# ---------------------------------------------------------------------------
# Eq. 4, Eq. 5, Eq. 1: geometry and compositing closed forms

def _single(mu, q, s, th, eta, tau, o, rgb):
    K = len(s)
    f = lambda a: np.asarray(a, np.float32)
    return synth.Scene(f([mu]), f([q]), f([s]), f([th]), f([eta]), f([tau]), f([o]), f([rgb]), -1)


def _front_uv(cam, mu, x, y):
    # camera_front: world axes = camera axes, eye at (0.5, 0.5, -1.5); the
    # plane z = mu_z is met at depth mu_z + 1.5, linearly in pixel coordinates
    z = mu[2] + 1.5
    u = 0.5 + z * (x + 0.5 - cam.cx) / cam.fx - mu[0]
    v = 0.5 + z * (y + 0.5 - cam.cy) / cam.fy - mu[1]
    return u, v


def test_fronto_parallel_single_primitive_image():
    cam = synth.camera_front(48, 40)
    mu = [0.52, 0.47, 0.3]
    su, sv = 0.05, 0.03
    sc = _single(mu, [1, 0, 0, 0], [su, sv, su, sv], [0, math.pi / 2, math.pi, 3 * math.pi / 2],
                 0.0, 0.0, 0.85, [0.9, 0.2, 0.4])
    bg = (0.1, 0.3, 0.05)
    opt = O.Options(alpha_min=1e-30, T_min=0.0, lowpass_sl=0.0, bg=bg)
    img = O.render(sc, cam, opt)["rgb"]
    mu32 = np.float32(mu).astype(np.float64)
    o = float(np.float32(0.85))
    col = np.float32([0.9, 0.2, 0.4]).astype(np.float64)
    s32 = np.float32([su, sv]).astype(np.float64)
    for y in range(cam.height):
        for x in range(cam.width):
            u, v = _front_uv(cam, mu32, x, y)
            a = min(o * math.exp(-0.5 * (u * u / s32[0] ** 2 + v * v / s32[1] ** 2)), 0.99)
            ref = a * col + (1 - a) * np.array(bg)
            np.testing.assert_allclose(img[:, y, x], ref, atol=1e-9)


def test_two_layers_closed_form_and_depth_order():
    cam = synth.camera_front(16, 16)
    far = [0.5, 0.5, 0.6]
    near = [0.5, 0.5, 0.2]
    th = [0, math.pi / 2, math.pi, 3 * math.pi / 2]
    s_big = [5.0] * 4   # nearly flat over the image
    f = lambda a: np.asarray(a, np.float32)
    sc = synth.Scene(f([far, near]), f([[1, 0, 0, 0]] * 2), f([s_big] * 2), f([th] * 2), f([0, 0]), f([0, 0]),
                     f([0.6, 0.3]), f([[1, 0, 0], [0, 0, 1]]), -1)
    opt = O.Options(alpha_min=1e-30, T_min=0.0, lowpass_sl=0.0, bg=(0, 1, 0))
    img = O.render(sc, cam, opt)["rgb"]
    for (x, y) in [(0, 0), (8, 8), (15, 3)]:
        a = []
        for k, mu in enumerate([far, near]):
            u, v = _front_uv(cam, np.float32(mu).astype(np.float64), x, y)
            a.append(float(np.float32([0.6, 0.3][k])) * math.exp(-(u * u + v * v) / (2 * 25.0)))
        a_far, a_near = a
        # the nearer primitive (index 1) is composited first
        ref = a_near * np.array([0, 0, 1]) + (1 - a_near) * (a_far * np.array([1, 0, 0]) +
                                                            (1 - a_far) * np.array([0, 1, 0]))
        np.testing.assert_allclose(img[:, y, x], ref, atol=1e-12)


def test_weights_sum_and_transmittance_monotone():
    sc = synth.scene_plain(300, 8, seed=11)
    cam = synth.camera_front(32, 32)
    opt = O.Options()
    out = O.render(sc, cam, opt)
    T = out["T"]
    assert np.all(T > 0) and np.all(T <= 1)
    # white colours, black background: C = sum of weights = 1 - T_final
    white = sc.copy()
    white.color[:] = 1.0
    img = O.render(white, cam, opt)["rgb"]
    np.testing.assert_allclose(img[0], 1.0 - T, atol=1e-12)
    # per pixel the sorted depths increase and T decreases
    for (x, y) in [(16, 16), (5, 20), (25, 7)]:
        idx, t, a, nc = O.contributors(sc, cam, opt, x, y)
        assert np.all(np.diff(t) >= 0)
        Ts = np.cumprod(np.concatenate([[1.0], 1 - a[:nc]]))
        assert np.all(np.diff(Ts) <= 0)
        assert Ts[-1] == pytest.approx(T[y, x], rel=1e-12)


def test_early_termination_count():
    # 30 identical fronto-parallel layers of constant alpha a: the stop comes
    # before the first layer j with (1 - a)^(j + 1) < T_min
    cam = synth.camera_front(8, 8)
    n = 30
    f = lambda v: np.asarray(v, np.float32)
    mu = [[0.5, 0.5, 0.1 + 0.02 * i] for i in range(n)]
    th = [0, math.pi / 2, math.pi, 3 * math.pi / 2]
    sc = synth.Scene(f(mu), f([[1, 0, 0, 0]] * n), f([[1e3] * 4] * n), f([th] * n), f([0] * n), f([0] * n),
                     f([0.4] * n), f([[1, 1, 1]] * n), -1)
    opt = O.Options(T_min=1e-4, lowpass_sl=0.0)
    out = O.render(sc, cam, opt)
    a = float(np.float32(0.4))
    expect = next(j for j in range(n) if (1 - a) ** (j + 1) < 1e-4)
    assert np.all(out["n_contrib"] == expect)


def test_filter_peaks_at_projected_centre_and_widens_with_tilt():
    # a primitive with a vanishing kernel (tiny scales) shows only the low-pass
    # filter of Eq. 10: value o at the projected centre, and a width that
    # grows as 1 / |cos| of the view angle.
    cam = synth.camera_front(64, 64)
    th = [0, math.pi / 2, math.pi, 3 * math.pi / 2]
    mu = [0.5, 0.5, 0.5]    # projects to the image centre (32, 32)
    opt = O.Options(alpha_min=1e-30, T_min=0.0, lowpass_sl=1.5, alpha_max=0.999)
    vals = []
    for beta in (0.0, 1.0):
        q = [math.cos(beta / 2), math.sin(beta / 2), 0, 0]           # tilt about x
        sc = _single(mu, q, [1e-5] * 4, th, 0.0, 0.0, 0.5, [1, 1, 1])
        ok, a_c, _ = O.pair(sc, 0, cam, opt, 31, 31)                 # offset (-0.5, -0.5)
        ok2, a_o, _ = O.pair(sc, 0, cam, opt, 33, 31)                # offset (1.5, -0.5)
        assert ok and ok2
        vals.append((a_c, a_o))
    o = float(np.float32(0.5))
    for a_c, a_o in vals:
        assert a_o < a_c <= o
    # ln(f/o) scales with cos^2 of the view angle at the pixel; the ratio
    # between the tilted and the fronto-parallel case is cos^2(tilted)/cos^2(front)
    d1 = np.array([(33.5 - 32) / cam.fx, (31.5 - 32) / cam.fy, 1.0])
    from scipy.spatial.transform import Rotation
    q32 = np.float32([math.cos(0.5), math.sin(0.5), 0, 0]).astype(np.float64)
    n_t = Rotation.from_quat([q32[1], q32[2], q32[3], q32[0]]).as_matrix()[:, 2]
    cos_f = 1 / np.linalg.norm(d1)
    cos_t = abs(d1 @ n_t) / np.linalg.norm(d1)
    r = math.log(vals[1][1] / o) / math.log(vals[0][1] / o)
    assert r == pytest.approx(cos_f ** 2 / cos_t ** 2, rel=1e-9)


# ---------------------------------------------------------------------------
# reverse mode against FP64 central finite differences

def _loss_fd(scene, cam, opt, gimg, name, index, h):
    vals = []
    for sgn in (1, -1):
        sc = scene.copy()
        arr = getattr(sc, name).astype(np.float64)
        arr[index] += sgn * h
        setattr(sc, name, arr)
        img = O.render(sc, cam, opt)["rgb"]
        vals.append(float(np.sum(img * gimg)))
    return (vals[0] - vals[1]) / (2 * h)


@pytest.mark.parametrize("sh_degree,sl", [(3, 0.7071), (-1, 0.0)])
def test_backward_matches_central_differences(sh_degree, sl):
    sc, cam = synth.scene_layers(n=64, K=8, seed=3100, sh_degree=sh_degree)
    # keep the float32 values exactly and differentiate in float64 around them
    sc = synth.Scene(**{k: v.astype(np.float64) for k, v in sc.arrays().items()}, sh_degree=sc.sh_degree)
    opt = O.Options(alpha_min=1e-20, T_min=0.0, lowpass_sl=sl)
    rng = np.random.default_rng(9)
    gimg = rng.standard_normal((3, cam.height, cam.width))
    grads = O.render_backward(sc, cam, opt, gimg)
    prims = rng.choice(sc.n, size=6, replace=False)
    checked = 0
    for name in ("mu", "quat", "scale", "theta", "eta", "tau", "opacity", "color"):
        arr = getattr(sc, name)
        for i in prims:
            sub = np.ndindex(arr.shape[1:]) if arr.ndim > 1 else [()]
            for j in sub:
                index = (i,) + tuple(j)
                if name == "color" and arr.ndim == 3 and j[0] > 4:
                    continue   # a few SH coefficients suffice (all share one code path)
                h = 1e-6 * max(1.0, abs(arr[index]))
                fd = _loss_fd(sc, cam, opt, gimg, name, index, h)
                an = grads[name][index]
                assert an == pytest.approx(fd, rel=2e-5, abs=2e-7 * (1 + abs(fd))), (name, index, an, fd)
                checked += 1
    assert checked > 100


# ---------------------------------------------------------------------------
# the paper's cache-sorting (Sec. 4.4 "Cache Sorting", supplementary
# Algorithm 1) as an alternative compositing order

def _literal(opt, cache_len=8):
    import dataclasses
    return dataclasses.replace(opt, order_mode=1, cache_len=cache_len)


def test_cache_sort_with_a_long_cache_is_the_exact_order():
    scene = synth.scene_clustered(1500, 8, seed=2200, n_clusters=6, sh_degree=-1)
    cam = synth.camera_front(40, 32)
    opt = O.Options()
    exact = O.render(scene, cam, opt)
    lit = O.render(scene, cam, _literal(opt, cache_len=100000))
    np.testing.assert_array_equal(exact["rgb"], lit["rgb"])
    np.testing.assert_array_equal(exact["T"], lit["T"])


def test_cache_sort_order_matches_an_independent_simulation():
    import bisect
    scene = synth.scene_clustered(1500, 8, seed=2201, n_clusters=6, sh_degree=-1)
    cam = synth.camera_front(40, 32)
    opt = O.Options()
    w2c = np.asarray(cam.world_to_cam, np.float64).reshape(3, 4)
    zc = np.asarray(scene.mu, np.float64) @ w2c[2, :3] + w2c[2, 3]
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(30):
        px, py = int(rng.integers(0, 40)), int(rng.integers(0, 32))
        idx, t, _, _ = O.contributors(scene, cam, opt, px, py)          # exact (r_t, index) order
        lidx, _, _, _ = O.contributors(scene, cam, _literal(opt, 2), px, py)
        rank = {int(i): k for k, i in enumerate(idx)}                     # position in the exact order
        pre = sorted(idx, key=lambda i: (zc[i], i))                       # pre-sort by centre depth
        cache, out = [], []
        for i in pre:
            bisect.insort(cache, rank[int(i)])
            if len(cache) > 2:
                out.append(int(idx[cache.pop(0)]))
        out += [int(idx[k]) for k in cache]
        assert out == [int(i) for i in lidx]
        checked += len(out) > 2
    assert checked >= 8     # pixels whose cache overflowed


def test_cache_sort_weights_sum_to_one_minus_T():
    scene = synth.scene_clustered(1500, 8, seed=2202, n_clusters=6, sh_degree=-1)
    scene.color[:] = 1.0                                                 # white: C = sum of weights
    cam = synth.camera_front(32, 24)
    opt = _literal(O.Options(bg=(0.0, 0.0, 0.0)), cache_len=2)
    r = O.render(scene, cam, opt)
    np.testing.assert_allclose(r["rgb"][0], 1.0 - r["T"], atol=1e-12)
