"""Pins of the oracle's paper-culling mode (Sec. 4.4, Eq. 11 - Eq. 12 as
printed): the endpoint radius 3 s for o = 1, tau = 0 (the "3-sigma" of
Eq. 11 without the factor 2), tiles kept exactly where the polygon meets
them (checked against a dense sampling of the polygon), and culling only
ever removes contributors."""
import math

import numpy as np
import pytest

from oracle import drk_oracle as O
from paper_2412_11752_gb300 import synth


def _one_primitive(mu, s, K=8):
    f = lambda a: np.asarray(a, np.float64)
    return synth.Scene(mu=f([mu]), quat=f([[1.0, 0, 0, 0]]), scale=f([[s] * K]),
                       theta=f([2 * np.pi * np.arange(K) / K]), eta=f([0.0]), tau=f([0.0]), opacity=f([1.0]),
                       color=f([[1.0, 1.0, 1.0]]), sh_degree=-1)


def test_paper_culling_keeps_exactly_the_tiles_the_3s_polygon_meets():
    cam = synth.camera_front(96, 96)
    z = 2.0                                   # depth of the plane z = 0.5 from the camera at z = -1.5
    s = 0.1
    # centre projected to continuous pixel coordinates (44, 40)
    X = (44.0 - cam.cx) * z / cam.fx + 0.5
    Y = (40.0 - cam.cy) * z / cam.fy + 0.5
    scene = _one_primitive([X, Y, 0.5], s)
    opt = O.Options(lowpass_sl=0.0)
    exact = O.render(scene, cam, opt)
    paper = O.render(scene, cam, O.Options(lowpass_sl=0.0, cull_paper=1))
    assert not np.any(paper["flags"] & O.FLAG_CULL)
    # tiles meeting the regular octagon of circumradius 3 s (in pixels 3 s f / z)
    R = 3 * s * cam.fx / z
    ang = 2 * np.pi * np.arange(8) / 8
    vx, vy = 44.0 + R * np.cos(ang), 40.0 + R * np.sin(ang)
    met = set()
    for a in range(8):
        b = (a + 1) % 8
        for u in np.linspace(0, 1, 400):
            for w in np.linspace(0, 1, 40):       # triangle (centre, v_a, v_b), dense
                x = 44.0 + w * ((1 - u) * (vx[a] - 44.0) + u * (vx[b] - 44.0))
                y = 40.0 + w * ((1 - u) * (vy[a] - 40.0) + u * (vy[b] - 40.0))
                # a tile's quad spans its corner pixel centres: continuous
                # [16 t + 0.5, 16 t + 15.5]; points between tiles meet neither
                tx, ty = int((x - 0.5) // 16), int((y - 0.5) // 16)
                if (x - 0.5) - 16 * tx <= 15 and (y - 0.5) - 16 * ty <= 15:
                    met.add((tx, ty))
    ys, xs = np.mgrid[0:96, 0:96]
    kept = np.array([[(x // 16, y // 16) in met for x in range(96)] for y in range(96)])
    np.testing.assert_array_equal(paper["rgb"][0][kept], exact["rgb"][0][kept])
    assert np.all(paper["rgb"][0][~kept] == 0.0)
    # the lost contributions lie between the 3 s polygon and the alpha_min
    # circle of radius sqrt(18) s
    lost = (~kept) & (exact["rgb"][0] > 0)
    assert lost.sum() > 0
    r = np.hypot(xs + 0.5 - 44.0, ys + 0.5 - 40.0)[lost] * z / cam.fx
    assert r.min() > 3 * s * math.cos(math.pi / 8) - 1e-9 and r.max() <= math.sqrt(18) * s + 1e-9


def test_paper_culling_only_removes_contributors():
    scene = synth.scene_plain(400, 8, seed=5201)
    cam = synth.camera_front(48, 48)
    e_opt, p_opt = O.Options(), O.Options(cull_paper=1)
    removed = 0
    for x, y in ((3, 5), (17, 30), (24, 24), (40, 11), (47, 47), (8, 40)):
        ie, _, _, _ = O.contributors(scene, cam, e_opt, x, y)
        ip, _, _, _ = O.contributors(scene, cam, p_opt, x, y)
        assert set(ip) <= set(ie)
        # the kept ones keep their order
        assert list(ip) == [i for i in ie if i in set(ip)]
        removed += len(ie) - len(ip)
    assert removed > 0
