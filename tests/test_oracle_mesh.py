"""Pins of the mesh conversion oracle (Sec. 5.4 and the supplementary
"Converting Mesh to DRK") and of the oracle's depth and normal images:
the converted kernel evaluated on the polygon's vertices, edges, inside and
outside; the frame and quaternion against the renderer oracle's rotation
and scipy; the extra endpoints' placement; rejections; a converted square
rendered fronto-parallel; closed forms of depth and normal for layers."""
import math

import numpy as np
import pytest

from oracle import drk_mesh_oracle as M
from oracle import drk_oracle as O
from paper_2412_11752_gb300 import synth


def _local(p, V, face):
    """(u, v) of world points in the converted DRK's frame."""
    R = O.rotation(p["quat"])
    return (np.asarray(V, np.float64) - p["mu"]) @ R[:, :2]


def _alpha(p, uv):
    return np.array([O.kernel_uv(p["scale"], p["theta"], p["eta"], p["tau"], p["opacity"], u, v) for u, v in uv])


def _polygon(m, r=1.0, sx=1.0, sy=0.6, rot=0.3, tilt=(0.2, -0.4, 0.9), centre=(0.3, -0.2, 2.0)):
    ang = rot + 2 * np.pi * np.arange(m) / m
    loc = np.stack([r * sx * np.cos(ang), r * sy * np.sin(ang), np.zeros(m)], axis=1)
    n = np.asarray(tilt, np.float64) / np.linalg.norm(tilt)
    a = np.cross(n, [1.0, 0, 0])
    a /= np.linalg.norm(a)
    b = np.cross(n, a)
    R = np.stack([a, b, n], axis=1)
    return loc @ R.T + np.asarray(centre), n


@pytest.mark.parametrize("m,K", [(3, 3), (3, 8), (4, 4), (4, 8), (6, 16)])
def test_converted_kernel_has_the_polygon_as_its_half_contour(m, K):
    V, n = _polygon(m)
    face = np.arange(m)
    opt = M.MeshOptions(K=K, tau=0.95, opacity=0.9)
    p, st = M.convert_face(V, face, np.ones(3), opt)
    assert st == 0
    uv = _local(p, V, face)
    # on the vertices and on points along every edge: Psi = 1/2
    edge = np.concatenate([V[j] + (V[(j + 1) % m] - V[j]) * t for j in range(m) for t in (0.0, 0.21, 0.5, 0.87)]
                          ).reshape(-1, 3)
    np.testing.assert_allclose(_alpha(p, _local(p, edge, face)), 0.5 * 0.9, rtol=1e-10)
    # centre: g = 1, Psi(1) = 1
    assert _alpha(p, [(0.0, 0.0)])[0] == pytest.approx(0.9, rel=1e-12)
    # scaled copies of the polygon inside and outside
    assert np.all(_alpha(p, 0.97 * uv) > 0.45) and np.all(_alpha(p, 1.03 * uv) < 0.45)
    # the frame: R_z is the face normal, the vertices lie in the plane
    R = O.rotation(p["quat"])
    assert abs(abs(R[:, 2] @ n) - 1.0) < 1e-12
    np.testing.assert_allclose((V - p["mu"]) @ R[:, 2], 0.0, atol=1e-12)
    np.testing.assert_allclose(p["mu"], V.mean(axis=0), rtol=1e-14)


def test_edge_density_exp_minus_half_puts_endpoints_on_the_vertices():
    V, _ = _polygon(5)
    p, st = M.convert_face(V, np.arange(5), np.ones(3), M.MeshOptions(K=5, edge_density=math.exp(-0.5), tau=0.0))
    uv = _local(p, V, np.arange(5))
    np.testing.assert_allclose(np.linalg.norm(uv, axis=1), p["scale"], rtol=1e-12)
    np.testing.assert_allclose(_alpha(p, uv), math.exp(-0.5), rtol=1e-10)   # tau = 0: Psi is the identity


def test_extra_endpoints_round_robin_on_the_edges():
    pts = np.array([[0.0, 0.0], [3.0, 0.0], [0.0, 2.0]])
    E = M.face_endpoints(3, 8, pts)
    assert len(E) == 8
    # 5 extra endpoints: edges 0 and 1 receive 2, edge 2 receives 1, evenly spaced
    np.testing.assert_allclose(E[:4], [[0, 0], [1, 0], [2, 0], [3, 0]], atol=1e-15)
    np.testing.assert_allclose(E[4:6], [[2, 2 / 3], [1, 4 / 3]], atol=1e-15)
    np.testing.assert_allclose(E[6:], [[0, 2], [0, 1]], atol=1e-15)


def test_quaternion_from_frame_matches_rotation_and_scipy():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rs = Rot.random(50, random_state=3)
    for r in rs:
        Rm = r.as_matrix()
        q = M.quat_from_matrix(Rm)
        assert q[0] >= 0 and abs(np.linalg.norm(q) - 1) < 1e-14
        np.testing.assert_allclose(O.rotation(q), Rm, atol=1e-12)
        xyzw = r.as_quat()
        ref = np.array([xyzw[3], *xyzw[:3]])
        np.testing.assert_allclose(q, ref if ref[0] >= 0 else -ref, atol=1e-12)


def test_rejected_faces():
    V = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 1, 0], [1, 1, 0], [0.5, 0.2, 0]], np.float64)
    opt = M.MeshOptions(K=4)
    assert M.convert_face(V, np.array([0, 1, 2, -1]), np.ones(3), opt)[1] == 1      # collinear
    assert M.convert_face(V, np.array([0, 1, 9, -1]), np.ones(3), opt)[1] == 1      # index out of range
    assert M.convert_face(V, np.array([0, -1, 1, 3]), np.ones(3), opt)[1] == 1      # padding inside the row
    assert M.convert_face(V, np.array([0, 1, -1, -1]), np.ones(3), opt)[1] == 1     # two vertices
    # a dart: the vertex mean lies outside the quad, the angles do not increase
    assert M.convert_face(V, np.array([0, 1, 5, 3]), np.ones(3), M.MeshOptions(K=4))[1] == 2
    p, st = M.convert_face(V, np.array([0, 1, 4, 3]), np.ones(3), opt)              # the unit square
    assert st == 0 and p["opacity"] == 1.0


def test_converted_square_renders_as_a_square():
    # a 0.8 x 0.8 square facing camera_front at depth 2.0: its image is the
    # projected square, sharp to within a pixel
    cam = synth.camera_front(64, 64)
    V = np.array([[0.1, 0.1, 0.5], [0.1, 0.9, 0.5], [0.9, 0.9, 0.5], [0.9, 0.1, 0.5]])
    p, st = M.convert_face(V, np.arange(4), np.array([0.2, 0.6, 1.0]),
                           M.MeshOptions(K=4, tau=0.95, ambient=1.0, diffuse=0.0))
    assert st == 0
    scene = synth.Scene(**{k: np.asarray(v, np.float64)[None] if np.ndim(v) else np.array([v], np.float64)
                           for k, v in p.items()}, sh_degree=-1)
    opt = O.Options(lowpass_sl=0.0)
    img = O.render(scene, cam, opt)["rgb"]
    # pixel centres of the projected square: x = fx (X - 0.5) / 2 + cx
    xs = (np.arange(64) + 0.5 - cam.cx) / cam.fx * 2.0 + 0.5
    inside_x = (xs > 0.1) & (xs < 0.9)
    dist = np.minimum(np.abs(xs - 0.1), np.abs(xs - 0.9)) * cam.fx / 2.0      # pixels to the nearest edge
    far = dist[:, None] > 1.0
    far = far & far.T
    inside = inside_x[:, None] & inside_x[None, :]
    a = img[2] / 1.0                                     # blue channel = alpha
    assert np.all(a[inside & far] > 0.97)
    assert np.all(a[~inside & far] < 0.02)
    np.testing.assert_allclose(img[0][inside & far] / a[inside & far], 0.2, rtol=1e-12)


def test_depth_and_normal_closed_forms():
    # two fronto-parallel layers (the second tilted) at depths z1 < z2:
    # depth = a1 z1 + (1 - a1) a2 z2 at the centre pixel, normal towards -z
    cam = synth.camera_front(32, 32)
    p1, _ = M.convert_face(np.array([[0.0, 0.0, 0.3], [0.0, 1.0, 0.3], [1.0, 1.0, 0.3], [1.0, 0.0, 0.3]]),
                           np.arange(4), np.ones(3), M.MeshOptions(K=4, tau=0.0, opacity=0.4))
    c, s_ = math.cos(0.5), math.sin(0.5)
    tilt = np.array([[-0.5, -0.5, 0.0], [-0.5, 1.5, 0.0], [1.5, 1.5, 0.0], [1.5, -0.5, 0.0]]) - [0.5, 0.5, 0.0]
    rot = np.array([[c, 0, s_], [0, 1, 0], [-s_, 0, c]])
    V2 = tilt @ rot.T + [0.5, 0.5, 0.9]
    p2, _ = M.convert_face(V2, np.arange(4), np.ones(3), M.MeshOptions(K=4, tau=0.0, opacity=0.7))
    scene = synth.Scene(**{k: np.stack([np.atleast_1d(np.asarray(p1[k], np.float64)),
                                        np.atleast_1d(np.asarray(p2[k], np.float64))]) for k in p1}, sh_degree=-1)
    opt = O.Options(lowpass_sl=0.0)
    pix = np.array([[16, 16], [5, 20]], np.int32)
    depth, normal = O.render_aux_pixels(scene, cam, opt, pix)
    for q in range(len(pix)):
        idx, t, a, nc = O.contributors(scene, cam, opt, *pix[q])
        assert list(idx) == [0, 1] and nc == 2
        assert depth[q] == pytest.approx(a[0] * t[0] + (1 - a[0]) * a[1] * t[1], rel=1e-12)
        # normals towards the camera (-z side): layer 1 (0, 0, -1), layer 2 rotated
        n2 = rot @ np.array([0, 0, -1.0])
        want = a[0] * np.array([0, 0, -1.0]) + (1 - a[0]) * a[1] * n2
        np.testing.assert_allclose(normal[q], want, atol=1e-12)
        # layer 1 faces the camera: its r_t is the view depth 0.3 + 1.5 everywhere
        assert t[0] == pytest.approx(1.8, rel=1e-12)
