"""GPU forward parity: the CUDA path through the C ABI against the FP64 oracle."""
import math

import numpy as np
import pytest

from helpers import TOL_IMAGE, excluded, image_parity, oracle_options, rel_err
from oracle import drk_oracle as O
from paper_2412_11752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drk():
    from paper_2412_11752_gb300 import drk as D
    D.lib()
    return D


def render_gpu(drk, scene, cam, opt, **kw):
    ds = drk.DeviceScene.from_scene(scene, "cuda")
    rgb, T, n, st = drk.drk_render(ds, cam, opt, **kw)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), T.cpu().numpy(), n.cpu().numpy(), st


def check_full(drk, scene, cam, opt, max_over_strict=2, what=""):
    rgb, T, n, _ = render_gpu(drk, scene, cam, opt)
    ref = O.render(scene, cam, oracle_options(opt))
    image_parity(rgb, ref, max_over_strict, what or f"{cam.width}x{cam.height}")
    keep = ~excluded(ref["flags"])
    assert np.abs(T - ref["T"])[keep].max() <= TOL_IMAGE
    return rgb, ref


def test_plain_2k_128_full_image(drk):
    scene = synth.scene_plain(2000, 8, seed=1000)
    cam = synth.camera_front(128, 128)
    opt = drk.Options()
    rgb, ref = check_full(drk, scene, cam, opt)
    assert rgb.max() > 0.1          # the image is not empty


CULL_CASES = {
    "plain-k8": (lambda: synth.scene_plain(2000, 8, seed=1000), lambda: synth.camera_front(128, 128)),
    "plain-k3": (lambda: synth.scene_plain(600, 3, seed=53), lambda: synth.camera_front(80, 72)),
    "slab-k16": (lambda: synth.scene_slab(3000, 16, seed=80), lambda: synth.camera_front(64, 64)),
    "clustered": (lambda: synth.scene_clustered(3000, 8, seed=70, n_clusters=6),
                  lambda: synth.camera_lookat(96, 64, eye=(1.9, 0.3, -0.8), target=(0.5, 0.5, 0.5))),
}


@pytest.mark.parametrize("case", sorted(CULL_CASES))
def test_cull_levels_bitwise_identical(drk, case):
    scene, cam = CULL_CASES[case][0](), CULL_CASES[case][1]()
    outs = []
    for lvl in (drk.CULL_NONE, drk.CULL_RECT, drk.CULL_TILE):
        rgb, T, n, _ = render_gpu(drk, scene, cam, drk.Options(cull_level=lvl))
        outs.append((rgb, T, n, drk.default_context().stats()))
    for rgb, T, n, _ in outs[1:]:
        assert np.array_equal(rgb, outs[0][0]) and np.array_equal(T, outs[0][1]) and np.array_equal(n, outs[0][2])
    pairs = [s["n_pairs"] for *_, s in outs]
    assert pairs[0] > pairs[1] > pairs[2] > 0, pairs


def test_buffer_capacity_does_not_change_the_image(drk):
    # the depth-order heap is exact for any capacity: a small shared part
    # spills to the overflow column or, without room there, takes extra
    # passes over the list, never a different order
    scene = synth.scene_clustered(4000, 8, seed=2100, n_clusters=8)
    cam = synth.camera_front(96, 64)
    r16, T16, n16, _ = render_gpu(drk, scene, cam, drk.Options(kbuf_capacity=16, ovf_capacity=-1))
    seen = {}
    for cap, ovf in ((8, 0), (8, 3), (8, -1), (32, 0), (16, 1)):
        r, T, n, _ = render_gpu(drk, scene, cam, drk.Options(kbuf_capacity=cap, ovf_capacity=ovf))
        st = drk.default_context().stats()
        assert np.array_equal(r, r16) and np.array_equal(T, T16) and np.array_equal(n, n16), (cap, ovf)
        seen[(cap, ovf)] = (st["n_spills"], st["n_extra_passes"])
    assert seen[(8, 0)][0] > 0 and seen[(8, 0)][1] == 0      # spills, no extra pass
    assert seen[(8, 3)][0] > 0 and seen[(8, 3)][1] > 0       # column too small: both
    assert seen[(8, -1)][0] == 0 and seen[(8, -1)][1] > 0    # no column: passes only


@pytest.mark.parametrize("cap", [8, 16])
def test_statistics_switch_keeps_images_and_gradients(drk, cap):
    # the forward without statistics (drk_stats_enable 0) renders the same
    # image bit for bit and the backward over its records gives the same
    # gradients (up to the order of float atomics); its five statistics
    # read 0, and two renders with statistics count the same (8 shared
    # heap slots make this scene spill; 16 is the default capacity)
    scene = synth.scene_clustered(4000, 8, seed=2100, n_clusters=8)
    cam = synth.camera_front(96, 64)
    opt = drk.Options(kbuf_capacity=cap)
    ds = drk.DeviceScene.from_scene(scene, "cuda")
    dL = torch.from_numpy(np.random.default_rng(7).standard_normal((3, 64, 96)).astype(np.float32)).cuda()
    ctx = drk.Context(0)
    fields = ("n_evals", "n_geo_evals", "n_contrib_evals", "n_emitted", "n_spills")

    def run(on):
        ctx.stats_enable(on)
        rgb, T, n, st = drk.drk_render(ds, cam, opt, ctx=ctx, need_state=True)
        stats = ctx.stats()
        g = drk.drk_render_backward(ds, cam, opt, st, dL, ctx=ctx)
        torch.cuda.synchronize()
        st.free()
        return rgb.cpu().numpy(), T.cpu().numpy(), n.cpu().numpy(), {k: v.cpu().numpy() for k, v in g.items()}, stats

    try:
        a, b, c = run(True), run(False), run(True)
    finally:
        ctx.close()
    for x in (b, c):
        for i in range(3):
            assert np.array_equal(x[i], a[i])
        # two backward runs sum their float atomics in different orders, which
        # moves single elements with heavy cancellation (quat) by more than
        # 1e-4 of themselves; per tensor the difference stays near float
        # rounding, while records that differed would move it by far more
        for k, v in a[3].items():
            assert rel_err(x[3][k], v) <= 5e-4, (k, rel_err(x[3][k], v))
    assert all(a[4][f] == c[4][f] for f in fields), (a[4], c[4])
    assert all(a[4][f] > 0 for f in fields if f != "n_spills" or cap == 8), a[4]
    assert all(b[4][f] == 0 for f in fields), b[4]
    assert b[4]["n_pairs"] == a[4]["n_pairs"] and b[4]["n_extra_passes"] == a[4]["n_extra_passes"]


def test_gaussian_special_case_k4(drk):
    # K = 4 right angles, eta = 0, tau = 0: planar anisotropic Gaussians (Eq. 3)
    sc = synth.scene_plain(400, 4, seed=41)
    sc.theta[:] = np.float32([0, math.pi / 2, math.pi, 3 * math.pi / 2])
    sc.scale[:, 2] = sc.scale[:, 0]
    sc.scale[:, 3] = sc.scale[:, 1]
    sc.eta[:] = 0
    sc.tau[:] = 0
    check_full(drk, sc, synth.camera_front(64, 64), drk.Options())


@pytest.mark.parametrize("K", [3, 5, 12, 16])
def test_other_basis_counts(drk, K):
    scene = synth.scene_plain(600, K, seed=50 + K)
    check_full(drk, scene, synth.camera_front(80, 72), drk.Options())


@pytest.mark.parametrize("wh", [(37, 23), (100, 61), (1, 1), (17, 16)])
def test_ragged_image_sizes(drk, wh):
    scene = synth.scene_plain(500, 8, seed=60)
    check_full(drk, scene, synth.camera_front(*wh), drk.Options())


def test_sh_colour_and_background(drk):
    scene = synth.scene_clustered(3000, 8, seed=70, n_clusters=6)
    cam = synth.camera_lookat(96, 64, eye=(1.9, 0.3, -0.8), target=(0.5, 0.5, 0.5))
    # thin planar clusters: crossing planes give many FP32-undecidable depth
    # ties; those pixels are held to their float32 budget
    check_full(drk, scene, cam, drk.Options(bg=(0.2, 0.5, 0.1)))


def test_filter_off_and_sharp_edges(drk):
    # tau near 1: Psi's middle slope (1 + tau)/(1 - tau) ~ 200 amplifies the
    # float32 error of edge pixels; they are held to their float32 budget
    scene = synth.scene_slab(3000, 16, seed=80)
    check_full(drk, scene, synth.camera_front(64, 64), drk.Options(lowpass_sl=0.0))


def test_empty_scene(drk):
    scene = synth.scene_plain(0, 8, seed=1)
    rgb, T, n, _ = render_gpu(drk, scene, synth.camera_front(40, 30), drk.Options(bg=(0.25, 0.5, 1.0)))
    assert np.all(rgb[0] == np.float32(0.25)) and np.all(rgb[2] == 1.0)
    assert np.all(T == 1.0) and np.all(n == 0)


def test_deterministic(drk):
    scene = synth.scene_plain(2000, 8, seed=1000)
    cam = synth.camera_front(128, 128)
    a = render_gpu(drk, scene, cam, drk.Options())[0]
    b = render_gpu(drk, scene, cam, drk.Options())[0]
    assert np.array_equal(a, b)


def test_invalid_arguments_rejected_on_host(drk):
    scene = synth.scene_plain(10, 8, seed=1)
    ds = drk.DeviceScene.from_scene(scene, "cuda")
    cam = synth.camera_front(16, 16)
    with pytest.raises(drk.DrkError) as e:
        drk.drk_render(ds, cam, drk.Options(kbuf_capacity=12))
    assert e.value.code == 1
    with pytest.raises(drk.DrkError):
        drk.drk_render(ds, cam, drk.Options(alpha_max=1.0))
    t = ds.tensors()
    t["scale"] = t["scale"][:, :2].contiguous()
    t["theta"] = t["theta"][:, :2].contiguous()
    with pytest.raises(drk.DrkError):                      # K = 2 < 3
        drk.drk_render(drk.DeviceScene(**t, sh_degree=-1), cam, drk.Options())


@pytest.mark.parametrize("n,bits", [(0, 32), (1, 32), (2, 8), (10007, 32), (1 << 20, 32), (300000, 20), (4096, 13)])
def test_sort_pairs_matches_stable_sort(drk, n, bits):
    rng = np.random.default_rng(n + bits)
    keys = rng.integers(0, 2 ** bits, size=n, dtype=np.uint64).astype(np.uint32)
    if n > 100:
        keys[: n // 3] = keys[0]          # many equal keys: stability matters
    vals = np.arange(n, dtype=np.uint32)
    k_t = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    v_t = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    drk.drk_sort_pairs(k_t, v_t, bits)
    torch.cuda.synchronize()
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(k_t.cpu().numpy().view(np.uint32), keys[order])
    assert np.array_equal(v_t.cpu().numpy().view(np.uint32), vals[order])


def densest_tile(scene, cam):
    """Tile (tx, ty) holding the most projected primitive centres (plain
    pinhole projection, test side)."""
    M = cam.world_to_cam.astype(np.float64)
    pc = scene.mu.astype(np.float64) @ M[:, :3].T + M[:, 3]
    px = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
    py = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
    ok = (pc[:, 2] > 0) & (px >= 0) & (px < cam.width) & (py >= 0) & (py < cam.height)
    tx = (cam.width + 15) // 16
    tid = (py[ok] // 16).astype(int) * tx + (px[ok] // 16).astype(int)
    dense = int(np.bincount(tid).argmax())
    return dense % tx, dense // tx


def full_size_tiles(scene, cam, count=4):
    """The densest tile, a bottom edge tile (partial when the height is not a
    multiple of 16), a corner tile and the centre tile (the first `count`)."""
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    return [densest_tile(scene, cam), (tx // 3, ty - 1), (0, 0), (tx // 2, ty // 2)][:count]


def check_sampled(drk, workload, count, seed, max_over_strict, opt=None, tiles=4):
    """A full-size workload rendered on the GPU, checked on seeded pixels
    plus whole tiles against the oracle (brute force per pixel)."""
    sc_f, cam_f = synth.WORKLOADS[workload]
    scene, cam = sc_f(), cam_f()
    opt = opt or drk.Options()
    rgb, T, n, _ = render_gpu(drk, scene, cam, opt)
    stats = drk.default_context().stats()
    pix = synth.pixel_sample(cam.width, cam.height, count, seed=seed, tiles=full_size_tiles(scene, cam, tiles))
    ref = O.render_pixels(scene, cam, oracle_options(opt), pix)
    image_parity(rgb[:, pix[:, 1], pix[:, 0]], ref, max_over_strict, workload)
    keep = ~excluded(ref["flags"])
    assert np.abs(T[pix[:, 1], pix[:, 0]] - ref["T"])[keep].max() <= TOL_IMAGE
    print(f"{workload}: {stats['n_pairs']} pairs, {stats['n_evals']} evaluations, {stats['n_emitted']} composited, "
          f"{stats['n_spills']} heap spills, {stats['n_extra_passes']} extra passes")
    assert stats["n_pairs"] > 0 and stats["n_evals"] > 0
    return stats


def test_clustered_100k_1080p_sampled_pixels(drk):
    # the benchmark workload: 16384 seeded pixels plus four whole tiles
    check_sampled(drk, "clustered-100k-1080p", 16384, 2001, max_over_strict=8)


def test_train_300k_1600x1064_sampled_pixels(drk):
    check_sampled(drk, "train-300k-1600x1064", 4096, 3002, max_over_strict=10)


def test_slab_2m_k16_4k_sampled_pixels(drk):
    # the stress workload: 2M primitives, K = 16, hard edges, 3840 x 2160
    # (pair offsets in 64 bits; about 8e8 pairs)
    st = check_sampled(drk, "slab-2M-k16-4k", 768, 5001, max_over_strict=8, tiles=2)
    assert st["n_pairs"] > (1 << 29)


# ---------------------------------------------------------------------------
# the paper's cache-sorting (Sec. 4.4, supplementary Algorithm 1): an
# approximate order, checked against the oracle's version of the same order

@pytest.mark.parametrize("cap", [8, 16])
def test_cache_sort_order_matches_oracle(drk, cap):
    scene = synth.scene_clustered(3000, 8, seed=2300, n_clusters=8, sh_degree=-1)
    cam = synth.camera_front(64, 48)
    opt = drk.Options(order_mode=1, kbuf_capacity=cap)
    rgb, ref = check_full(drk, scene, cam, opt, max_over_strict=4)
    # the approximation is visible: it differs from the exact order somewhere
    exact = O.render(scene, cam, oracle_options(drk.Options()))
    assert np.abs(ref["rgb"] - exact["rgb"]).max() > 1e-3


def test_cache_sort_without_overflow_is_exact(drk):
    # with 30 primitives a 32-entry cache never overflows, so it composites
    # in exact order
    scene = synth.scene_plain(30, 8, seed=2301)
    cam = synth.camera_front(48, 48)
    lit, _, _, _ = render_gpu(drk, scene, cam, drk.Options(order_mode=1, kbuf_capacity=32))
    ex, _, _, _ = render_gpu(drk, scene, cam, drk.Options())
    np.testing.assert_array_equal(lit, ex)


def test_cache_sort_has_no_backward(drk):
    scene = synth.scene_plain(100, 8, seed=2302)
    ds = drk.DeviceScene.from_scene(scene, "cuda")
    with pytest.raises(drk.DrkError) as e:
        drk.drk_render(ds, synth.camera_front(16, 16), drk.Options(order_mode=1), need_state=True)
    assert e.value.code == 1


# ---------------------------------------------------------------------------
# the paper's tile culling as printed (Eq. 11 - Eq. 12): lossy, checked
# against the oracle applying the same rule

@pytest.mark.parametrize("K,seed,sh", [(8, 2310, -1), (5, 2311, -1), (12, 2312, 1)])
def test_paper_culling_matches_oracle(drk, K, seed, sh):
    scene = synth.scene_plain(1500, K, seed=seed, sh_degree=sh)
    cam = synth.camera_front(96, 80)
    opt = drk.Options(cull_level=drk.CULL_PAPER)
    rgb, ref = check_full(drk, scene, cam, opt)
    pairs_paper = drk.default_context().stats()["n_pairs"]
    render_gpu(drk, scene, cam, drk.Options())
    pairs_tile = drk.default_context().stats()["n_pairs"]
    assert pairs_paper < pairs_tile
    # lossy: the image differs from the exact one
    exact = O.render(scene, cam, oracle_options(drk.Options()))
    assert np.abs(ref["rgb"] - exact["rgb"]).max() > 1e-3
