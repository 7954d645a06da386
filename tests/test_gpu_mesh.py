"""GPU tests of the mesh conversion (Sec. 5.4 and the supplementary
"Converting Mesh to DRK") and of the depth and normal images: the converted
parameters against the FP64 mesh oracle, rejected faces, a converted
height-field wall rendered against the renderer oracle (colour, depth,
normal), and its coverage (the faces meet without gaps)."""
import numpy as np
import pytest

from helpers import excluded, image_parity, oracle_options
from oracle import drk_mesh_oracle as M
from oracle import drk_oracle as O
from paper_2412_11752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drk():
    from paper_2412_11752_gb300 import drk as D
    D.lib()
    return D


def _convert(drk, verts, faces, colors, mopt):
    sc, st = drk.mesh_to_drk(torch.from_numpy(verts).cuda(), torch.from_numpy(faces).cuda(),
                             torch.from_numpy(colors).cuda(), mopt)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in sc.tensors().items()}, st.cpu().numpy(), sc


def _oracle_mesh_options(mopt):
    f = lambda x: float(np.float32(x))
    return M.MeshOptions(K=mopt.K, edge_density=f(mopt.edge_density), tau=f(mopt.tau), opacity=f(mopt.opacity),
                         light=tuple(f(x) for x in mopt.light), ambient=f(mopt.ambient), diffuse=f(mopt.diffuse))


def _bad_faces(verts, face_size):
    """Faces the conversion must reject, appended to a mesh: (verts, faces,
    expected status)."""
    n = len(verts)
    extra = np.array([[0, 0, 5], [1, 0, 5], [2, 0, 5], [0, 1, 5], [0.5, 0.2, 5]], np.float32)
    v = np.concatenate([verts, extra])
    pad = lambda r: r + [-1] * (face_size - len(r))
    rows, want = [], []
    rows.append(pad([n, n + 1, n + 2])); want.append(1)                 # collinear
    rows.append(pad([n, n + 1, len(v) + 7])); want.append(1)            # index out of range
    if face_size >= 4:
        rows.append([n, -1, n + 1] + [n + 3] * (face_size - 3)); want.append(1)   # padding inside the row
        rows.append(pad([n, n + 1, n + 4, n + 3])); want.append(2)      # a dart
    rows.append(pad([n, n + 1])); want.append(1)                        # two vertices
    return v, np.asarray(rows, np.int32), want


@pytest.mark.parametrize("kind,K", [("quads", 4), ("quads", 8), ("tris", 3), ("tris", 16), ("polygons", 8)])
def test_mesh_conversion_matches_oracle(drk, kind, K):
    if kind == "polygons":
        verts, faces = synth.mesh_polygons(400, max_vertices=8, seed=7101)
    else:
        verts, faces = synth.mesh_heightfield(20, 14, seed=7001, triangles=(kind == "tris"))
    verts, bad, want_bad = _bad_faces(verts, faces.shape[1])
    faces = np.concatenate([faces, bad])
    colors = synth.mesh_colors(len(faces), seed=7201)
    mopt = drk.MeshOptions(K=K, tau=0.9, opacity=0.95, edge_density=0.5)
    got, st, _ = _convert(drk, verts, faces, colors, mopt)
    ref, rst = M.mesh_to_drk(verts.astype(np.float64), faces, colors.astype(np.float64), _oracle_mesh_options(mopt))
    np.testing.assert_array_equal(st, rst)
    assert list(st[-len(want_bad):]) == want_bad
    ok = st == 0
    assert ok.sum() >= len(faces) - len(want_bad)
    np.testing.assert_allclose(got["mu"][ok], ref["mu"][ok], rtol=1e-6, atol=1e-6)
    Rg = np.stack([O.rotation(q) for q in got["quat"][ok]])
    Rr = np.stack([O.rotation(q) for q in ref["quat"][ok]])
    np.testing.assert_allclose(Rg, Rr, atol=3e-5)
    np.testing.assert_allclose(got["theta"][ok], ref["theta"][ok], atol=3e-5)
    np.testing.assert_allclose(got["scale"][ok], ref["scale"][ok], rtol=3e-5)
    np.testing.assert_allclose(got["color"][ok], ref["color"][ok], rtol=1e-5, atol=1e-6)
    for k in ("eta", "tau", "opacity"):
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-7, err_msg=k)
    # rejected faces render nothing
    assert np.all(got["opacity"][~ok] == 0.0)


def test_mesh_options_rejected(drk):
    verts, faces = synth.mesh_heightfield(2, 2)
    colors = synth.mesh_colors(len(faces))
    for bad in (drk.MeshOptions(K=2), drk.MeshOptions(K=4, edge_density=1.0), drk.MeshOptions(tau=1.0),
                drk.MeshOptions(opacity=0.0), drk.MeshOptions(light=(0.0, 0.0, 0.0))):
        with pytest.raises(drk.DrkError) as e:
            _convert(drk, verts, faces, colors, bad)
        assert e.value.code == 1


def _wall(drk, nx, ny, K, tau, W, H, triangles=False):
    verts, faces = synth.mesh_heightfield(nx, ny, seed=7002, triangles=triangles)
    colors = synth.mesh_colors(len(faces), seed=7202)
    got, st, sc = _convert(drk, verts, faces, colors, drk.MeshOptions(K=K, tau=tau))
    assert np.all(st == 0)
    scene = synth.Scene(**{k: np.asarray(v, np.float32) for k, v in got.items()}, sh_degree=-1)
    return scene, sc, synth.camera_front(W, H)


@pytest.mark.parametrize("K,tau", [(4, 0.6), (8, 0.8)])
def test_converted_wall_renders_like_the_oracle_with_depth_and_normal(drk, K, tau):
    scene, sc, cam = _wall(drk, 12, 8, K, tau, 96, 64)
    opt = drk.Options()
    rgb, T, depth, normal = drk.drk_render_aux(sc, cam, opt)
    torch.cuda.synchronize()
    rgb, T, depth, normal = (x.cpu().numpy().astype(np.float64) for x in (rgb, T, depth, normal))
    oo = oracle_options(opt)
    ref = O.render(scene, cam, oo)
    rd, rn = O.render_aux(scene, cam, oo)
    image_parity(rgb, ref, 2, f"converted wall K={K}")
    ex = excluded(ref["flags"])
    assert ex.mean() < 0.1, ex.mean()
    keep = ~ex
    for c in range(3):
        assert np.abs(normal[c] - rn[c])[keep].max() <= 2e-4
    # depth: the colour's tolerance on weights that sum to at most 1, times the depth
    assert (np.abs(depth - rd)[keep] / np.maximum(rd[keep], 1.0)).max() <= 2e-4
    # the colour image is unchanged by asking for depth and normal
    plain, _, _, _ = drk.drk_render(sc, cam, opt)
    assert np.array_equal(plain.cpu().numpy(), rgb.astype(np.float32))


def test_converted_wall_is_closed(drk):
    # neighbouring triangles (planar, so a shared edge is the same segment in
    # both) meet on their Psi = 1/2 contours: the wall covers the image it
    # spans without gaps; seen head on its normal faces the camera and its
    # mean depth is the wall's depth.  (Non-planar quads are flattened onto
    # their own planes, so neighbours can leave sub-pixel cracks.)
    scene, sc, cam = _wall(drk, 24, 16, 3, 0.95, 192, 128, triangles=True)
    rgb, T, depth, normal = drk.drk_render_aux(sc, cam, drk.Options())
    torch.cuda.synchronize()
    T, depth, normal = T.cpu().numpy(), depth.cpu().numpy(), normal.cpu().numpy()
    # pixels well inside the wall's silhouette (it spans x in [-0.3, 1.3] and
    # y in [-0.1, 1.1] at a depth of about 2.1)
    xs = (np.arange(192) + 0.5 - cam.cx) / cam.fx * 2.1 + 0.5
    ys = (np.arange(128) + 0.5 - cam.cy) / cam.fy * 2.1 + 0.5
    inner = ((xs > -0.2) & (xs < 1.2))[None, :] & ((ys > 0.0) & (ys < 1.0))[:, None]
    assert np.median(T[inner]) < 0.02
    assert T[inner].max() < 0.3          # at worst two half-covered faces on an edge
    cov = 1.0 - T[inner]
    assert np.all(normal[2][inner] / cov < -0.9)
    zmean = depth[inner] / cov
    assert np.all(np.abs(zmean - 2.1) < 0.12)
