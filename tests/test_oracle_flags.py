"""Pins of the oracle's float32-undecidability flags: two coplanar
contributors have exactly equal r_t, so float32 may composite them in
either order; the pixel is flagged when exchanging them changes the
colour visibly, in the exact order and in the cache-sorting order, and not
when their colours are equal."""
import numpy as np

from oracle import drk_oracle as O
from paper_2412_11752_gb300 import synth


def _two_coplanar(c0, c1):
    f = lambda a: np.asarray(a, np.float64)
    K = 4
    return synth.Scene(mu=f([[0.5, 0.5, 0.5], [0.52, 0.49, 0.5]]), quat=f([[1.0, 0, 0, 0]] * 2),
                       scale=f([[0.2] * K] * 2), theta=f([2 * np.pi * np.arange(K) / K] * 2), eta=f([0.0, 0.0]),
                       tau=f([0.0, 0.0]), opacity=f([0.6, 0.6]), color=f([c0, c1]), sh_degree=-1)


def test_equal_depths_with_different_colours_are_flagged():
    cam = synth.camera_front(16, 16)
    pix = np.array([[8, 8]], np.int32)
    for mode in (0, 1):
        opt = O.Options(lowpass_sl=0.0, order_mode=mode, cache_len=8)
        idx, t, a, nc = O.contributors(_two_coplanar([1.0, 0.0, 0.0], [0.0, 0.0, 1.0]), cam, opt, 8, 8)
        assert len(idx) == 2 and t[0] == t[1]                  # the same plane: r_t exactly equal
        r = O.render_pixels(_two_coplanar([1.0, 0.0, 0.0], [0.0, 0.0, 1.0]), cam, opt, pix)
        assert r["flags"][0] & O.FLAG_DEPTH_TIE, mode
        same = O.render_pixels(_two_coplanar([0.3, 0.3, 0.3], [0.3, 0.3, 0.3]), cam, opt, pix)
        assert not same["flags"][0] & O.FLAG_DEPTH_TIE, mode
        # the pixel's float32 budget covers the exchange: composited in the
        # other order the colour moves by exactly a0 a1 |c0 - c1| (T = 1)
        swap = a[0] * a[1] * 1.0
        assert r["tol"][0] >= swap * (1 - 1e-9), (r["tol"][0], swap)
        assert same["tol"][0] < 1e-5


def test_budget_covers_an_undecidable_stop():
    # identical fronto-parallel layers: compositing stops before the first
    # layer whose T (1 - a) falls below T_min; with T_min set to that value
    # exactly the stop is undecidable and the budget must cover the colour
    # change of deciding it either way (one layer more or less)
    f = lambda v: np.asarray(v, np.float64)
    n, K = 6, 4
    sc = synth.Scene(mu=f([[0.5, 0.5, 0.3 + 0.05 * i] for i in range(n)]), quat=f([[1.0, 0, 0, 0]] * n),
                     scale=f([[0.3] * K] * n), theta=f([2 * np.pi * np.arange(K) / K] * n), eta=f([0.0] * n),
                     tau=f([0.0] * n), opacity=f([0.5] * n), color=f([[0.9, 0.1, 0.5]] * n), sh_degree=-1)
    cam = synth.camera_front(16, 16)
    pix = np.array([[8, 8]], np.int32)
    base = O.Options(lowpass_sl=0.0, T_min=0.0)
    idx, t, a, nc = O.contributors(sc, cam, base, 8, 8)
    T = np.cumprod(np.concatenate([[1.0], 1 - a]))
    stop = 3                                   # T_min exactly at T_3 (1 - a_3)
    opt = O.Options(lowpass_sl=0.0, T_min=float(T[stop] * (1 - a[stop])))
    r = O.render_pixels(sc, cam, opt, pix)
    assert r["flags"][0] & O.FLAG_T_MIN
    one_more = T[stop] * a[stop] * 0.9          # composite layer 3 too (bg = 0)
    assert r["tol"][0] >= one_more * (1 - 1e-9), (r["tol"][0], one_more)


def test_excluded_covers_every_undecidable_flag():
    from helpers import excluded, undecidable
    for f in (O.FLAG_T_MIN, O.FLAG_DEPTH_TIE, O.FLAG_STEEP, O.FLAG_CULL):
        assert excluded(np.array([f]))[0]
    for f in (O.FLAG_T_MIN, O.FLAG_DEPTH_TIE, O.FLAG_CULL):
        assert undecidable(np.array([f]))[0]
    assert not undecidable(np.array([O.FLAG_STEEP]))[0]       # continuous: within the budget
    assert not excluded(np.array([O.FLAG_ALPHA_MIN]))[0]      # informational only


# ---------------------------------------------------------------------------
# derivative branch points (FLAG_KINK): a composited alpha at a breakpoint of
# Psi (Eq. 9), at the max of kernel and filter (Eq. 10) or at the clamp
# alpha_max is continuous but not differentiable, so float32 may take the
# other one-sided gradient there

def _plane_uv(cam, mu, x, y):
    """(u, v) where the ray of pixel (x, y) meets the plane z = mu_z of a
    primitive with identity rotation (axes x, y), from the camera's own
    world-to-camera matrix, independently of the oracle."""
    M = np.asarray(cam.world_to_cam, np.float64)
    R, t = M[:, :3], M[:, 3]
    c = -R.T @ t
    d = R.T @ np.array([(x + 0.5 - cam.cx) / cam.fx, (y + 0.5 - cam.cy) / cam.fy, 1.0])
    s = (mu[2] - c[2]) / d[2]
    p = c + s * d - np.asarray(mu, np.float64)
    return p[0], p[1]


def _gaussian(mu, s, tau, o):
    # equal scales and eta = 0: g = exp(-r^2 / (2 s^2)) (Eq. 6, Eq. 8)
    f = lambda a: np.asarray(a, np.float64)
    K = 4
    return synth.Scene(mu=f([mu]), quat=f([[1.0, 0, 0, 0]]), scale=f([[s] * K]),
                       theta=f([2 * np.pi * np.arange(K) / K]), eta=f([0.0]), tau=f([tau]), opacity=f([o]),
                       color=f([[0.8, 0.3, 0.1]]), sh_degree=-1)


def test_kink_flag_at_a_breakpoint_of_psi():
    cam = synth.camera_front(16, 16)
    mu = (0.53, 0.47, 0.5)
    u, v = _plane_uv(cam, mu, 8, 8)
    r2 = u * u + v * v
    pix = np.array([[8, 8]], np.int32)
    opt = O.Options(lowpass_sl=0.0)
    for tau in (0.5, 0.95):
        for b in ((1 + tau) / 4, (3 - tau) / 4):
            s = np.sqrt(r2 / (-2.0 * np.log(b)))           # g = b at this pixel
            at = O.render_pixels(_gaussian(mu, s, tau, 0.8), cam, opt, pix)
            assert at["flags"][0] & O.FLAG_KINK, (tau, b)
            # one percent of scale away: g moves far beyond its float32 error
            off = O.render_pixels(_gaussian(mu, s * 1.01, tau, 0.8), cam, opt, pix)
            assert not off["flags"][0] & O.FLAG_KINK, (tau, b)
            # the image does not care: same colour to first order, no other flag
            assert not at["flags"][0] & (O.FLAG_T_MIN | O.FLAG_DEPTH_TIE)
    # tau = 0: Psi is the identity, no slope jump, no flag
    s = np.sqrt(r2 / (-2.0 * np.log(0.25)))
    flat = O.render_pixels(_gaussian(mu, s, 0.0, 0.8), cam, opt, pix)
    assert not flat["flags"][0] & O.FLAG_KINK


def test_kink_flag_at_the_filter_max_and_the_clamp():
    cam = synth.camera_front(16, 16)
    # the centre projects to the centre of pixel (8, 8): the filter there is
    # o, and the kernel at r = 0 is o Psi(1) = o (Eq. 10: equal branches)
    zc = 0.5 + 1.5
    mu = (0.5 + 0.5 * zc / cam.fx, 0.5 + 0.5 * zc / cam.fy, 0.5)
    pix = np.array([[8, 8], [11, 10], [11, 8]], np.int32)
    r = O.render_pixels(_gaussian(mu, 0.2, 0.0, 0.5), cam, O.Options(), pix)
    assert r["flags"][0] & O.FLAG_KINK
    assert not r["flags"][1] & O.FLAG_KINK      # (3, 2) px away: the filter is ~e^-13 o
    # on the u axis the polar angle is the basis angle theta_0 = 0: a sector
    # boundary, where the L1 term of Eq. 7 changes basis
    assert r["flags"][2] & O.FLAG_KINK
    # the clamp: opacity equal to alpha_max at the centre
    opt = O.Options(lowpass_sl=0.0, alpha_max=0.9)
    at = O.render_pixels(_gaussian(mu, 0.2, 0.0, 0.9), cam, opt, pix[:1])
    assert at["flags"][0] & O.FLAG_KINK
    below = O.render_pixels(_gaussian(mu, 0.2, 0.0, 0.85), cam, opt, pix[:1])
    assert not below["flags"][0] & O.FLAG_KINK


def test_grad_excluded_adds_the_kink_flag():
    from helpers import excluded, grad_excluded
    assert grad_excluded(np.array([O.FLAG_KINK]))[0]
    assert not excluded(np.array([O.FLAG_KINK]))[0]          # images are continuous there
    for f in (O.FLAG_T_MIN, O.FLAG_DEPTH_TIE, O.FLAG_STEEP, O.FLAG_CULL):
        assert grad_excluded(np.array([f]))[0]
