"""GPU reverse mode against the oracle's analytic (back-to-front) derivative.

The oracle's derivative is itself pinned to FP64 central differences
(test_oracle_pins.py); here the CUDA backward, which replays the forward
front to back, must agree with it per parameter tensor."""
import numpy as np
import pytest

from helpers import TOL_GRAD_REL, grad_excluded, oracle_options, rel_err
from oracle import drk_oracle as O
from paper_2412_11752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ("mu", "quat", "scale", "theta", "eta", "tau", "opacity", "color")


@pytest.fixture(scope="module")
def drk():
    from paper_2412_11752_gb300 import drk as D
    D.lib()
    return D


def compare_grads(drk, scene, cam, opt, seed=0, names=NAMES, tol=TOL_GRAD_REL):
    ds = drk.DeviceScene.from_scene(scene, "cuda")
    rgb, T, n, st = drk.drk_render(ds, cam, opt, need_state=True)
    oopt = oracle_options(opt)
    ref_f = O.render(scene, cam, oopt)
    w = np.random.default_rng(seed).standard_normal((3, cam.height, cam.width))
    w[:, grad_excluded(ref_f["flags"])] = 0.0      # no dL on float32-undecidable pixels
    g = drk.drk_render_backward(ds, cam, opt, st, torch.from_numpy(w.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    st.free()
    ref = O.render_backward(scene, cam, oopt, w)
    report = _compare_tensors(g, ref, names, tol, f"{cam.width}x{cam.height}")
    return report


def _compare_tensors(g, ref, names, tol, what, rel_elem=None):
    """Per tensor: relative L2 error <= tol, and every element within
    1e-3 max|ref| + e |ref|, e = 1e-3, or per primitive rel_elem when given."""
    report = {}
    for k in names:
        a = g[k].cpu().numpy().astype(np.float64)
        b = ref[k]
        r = rel_err(a, b)
        report[k] = r
        assert np.all(np.isfinite(a)), k
        assert r <= tol, f"{what} {k}: relative error {r:.2e} (all: {report})"
        e = 1e-3 if rel_elem is None else rel_elem.reshape((-1,) + (1,) * (b.ndim - 1))
        bound = 1e-3 * np.abs(b).max() + e * np.abs(b) + 1e-7
        worst = np.max(np.abs(a - b) - bound)
        assert worst <= 0, f"{what} {k}: elementwise excess {worst:.2e}"
    print(f"{what}: gradient relative errors " + ", ".join(f"{k} {v:.1e}" for k, v in report.items()))
    return report


def alpha_conditioning(scene, cam, oopt, pixels) -> np.ndarray:
    """Per primitive: the largest relative float32 error, by the oracle's
    error model (test_oracle_error_model.py pins it), of its composited
    alphas in the given pixels (0 where it has none).  A primitive seen only
    through pairs whose alpha float32 resolves to 1 % has a gradient that
    float32 resolves to about as much: Psi's middle slope (1 + tau)/(1 - tau)
    of Eq. 9 (up to 199 at tau = 0.99), grazing rays and narrow sectors
    amplify the rounding of g, r_t and the polar angle."""
    import concurrent.futures as cf
    import os

    def one(xy):
        idx, t, a, nc = O.contributors(scene, cam, oopt, int(xy[0]), int(xy[1]))
        return idx[:nc], np.repeat(np.array([xy], np.int32), nc, axis=0)

    rho = np.zeros(scene.n)
    # one pixel per call; the oracle library releases the interpreter lock
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        res = list(ex.map(one, [tuple(p) for p in pixels]))
    ii = [r[0] for r in res]
    pp = [r[1] for r in res]
    ii = np.concatenate(ii)
    r = O.pairs(scene, cam, oopt, ii, np.concatenate(pp))
    ratio = np.where(r["alpha"] > 0, r["dalpha"] / np.maximum(r["alpha"], 1e-300), 0.0)
    np.maximum.at(rho, ii, ratio)
    return rho


def compare_grads_sampled(drk, workload, count, seed, tiles, opt=None, conditioned=False):
    """Backward of a full-size workload with dL nonzero only on seeded pixels
    plus whole tiles, against the oracle's back-to-front derivative of those
    pixels.  Pixels the oracle flags get dL = 0: a float32-undecidable stop,
    depth tie or culling decision, alphas whose float32 error the budget
    lets exceed half the image tolerance (hard edges), or a composited
    alpha within float32 rounding of a point where its derivative changes
    branch (Psi's breakpoints, the max of Eq. 10, the clamp)."""
    from test_gpu_render import full_size_tiles
    sc_f, cam_f = synth.WORKLOADS[workload]
    scene, cam = sc_f(), cam_f()
    opt = opt or drk.Options()
    ds = drk.DeviceScene.from_scene(scene, "cuda")
    rgb, T, n, st = drk.drk_render(ds, cam, opt, need_state=True)
    oopt = oracle_options(opt)
    pix = synth.pixel_sample(cam.width, cam.height, count, seed=seed, tiles=full_size_tiles(scene, cam, tiles))
    keep = ~grad_excluded(O.render_pixels(scene, cam, oopt, pix)["flags"])
    pk = pix[keep]
    wpix = np.random.default_rng(seed + 1).standard_normal((pk.shape[0], 3))
    w = np.zeros((3, cam.height, cam.width), np.float32)
    w[:, pk[:, 1], pk[:, 0]] = wpix.T
    g = drk.drk_render_backward(ds, cam, opt, st, torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    st.free()
    stats = drk.default_context().stats()
    ref = O.render_backward_pixels(scene, cam, oopt, pk, w[:, pk[:, 1], pk[:, 0]].T.astype(np.float64))
    print(f"{workload}: {pk.shape[0]} of {pix.shape[0]} sampled pixels carry dL, "
          f"{stats['n_replay_evals']} replay evaluations")
    rel_elem = None
    if conditioned:
        # elementwise: each primitive to 1e-3 or to twice the float32
        # resolution of its alphas in these pixels, whichever is larger
        rho = alpha_conditioning(scene, cam, oopt, pk)
        rel_elem = np.maximum(1e-3, 2.0 * rho)
        print(f"{workload}: {int((rel_elem > 1e-3).sum())} primitives with alphas resolved to worse than 5e-4 "
              f"(largest relative float32 error {rho.max():.1e})")
    _compare_tensors(g, ref, NAMES, TOL_GRAD_REL, workload, rel_elem)
    return stats


def test_backward_clustered_100k_1080p_sampled(drk):
    compare_grads_sampled(drk, "clustered-100k-1080p", 2048, 2101, tiles=4)


def test_backward_train_300k_1600x1064_sampled(drk):
    compare_grads_sampled(drk, "train-300k-1600x1064", 1024, 3102, tiles=2)


def test_backward_slab_2m_k16_4k_sampled(drk):
    # the stress workload: 2M primitives, K = 16, sharpness near 1,
    # 3840 x 2160, about 8e8 pairs (64-bit pair offsets, the largest record
    # pool, exceeded here: most tiles take the exact replay); 128 seeded
    # pixels plus the densest tile carry dL.  Sharpness near 1 leaves some
    # alphas resolved by float32 to only about 1 %, so each primitive's
    # elements are held to the resolution of its alphas (per-tensor error
    # stays at 1e-3)
    st = compare_grads_sampled(drk, "slab-2M-k16-4k", 128, 5101, tiles=1, conditioned=True)
    print(f"slab-2M-k16-4k backward: {st['n_pairs']} pairs, {st['n_emitted']} composited, "
          f"{st['n_replay_evals']} replay evaluations")
    assert st["n_pairs"] > (1 << 29)


@pytest.mark.parametrize("chunks", [1, 6])
def test_backward_with_record_pool_overflow(drk, chunks):
    # a capped record pool sends tiles to the exact replay of the forward
    # traversal; the gradients stay the oracle's
    scene = synth.scene_clustered(2000, 8, seed=3200, n_clusters=5)
    cam = synth.camera_lookat(64, 64, eye=(1.5, -0.4, -1.0), target=(0.5, 0.5, 0.5))
    compare_grads(drk, scene, cam, drk.Options(record_chunks=chunks), seed=2)
    st = drk.default_context().stats()
    assert st["n_replay_evals"] > 0


def test_backward_layers_no_thresholds(drk):
    # the finite-difference sub-case: 64 primitives, 32 x 32, every pair
    # contributes (alpha_min 1e-20, T_min 0), opacity <= 0.95
    scene, cam = synth.scene_layers(64, 8, seed=3100)
    opt = drk.Options(alpha_min=1e-20, T_min=0.0)
    compare_grads(drk, scene, cam, opt)


def test_backward_layers_plain_rgb_filter_off(drk):
    scene, cam = synth.scene_layers(64, 8, seed=3101, sh_degree=-1)
    opt = drk.Options(alpha_min=1e-20, T_min=0.0, lowpass_sl=0.0)
    compare_grads(drk, scene, cam, opt)


def test_backward_default_thresholds_plain(drk):
    scene = synth.scene_plain(300, 8, seed=77)
    cam = synth.camera_front(64, 48)
    compare_grads(drk, scene, cam, drk.Options(), seed=1)


def test_backward_clustered_sh(drk):
    scene = synth.scene_clustered(2000, 8, seed=3200, n_clusters=5)
    cam = synth.camera_lookat(64, 64, eye=(1.5, -0.4, -1.0), target=(0.5, 0.5, 0.5))
    compare_grads(drk, scene, cam, drk.Options(), seed=2)


def test_backward_k16_small_buffer(drk):
    scene = synth.scene_slab(800, 16, seed=3300)
    cam = synth.camera_front(48, 48)
    compare_grads(drk, scene, cam, drk.Options(kbuf_capacity=8), seed=3)


def test_autograd_function_l1_loss(drk):
    scene = synth.scene_plain(300, 8, seed=78)
    cam = synth.camera_front(40, 40)
    opt = drk.Options()
    ds = drk.DeviceScene.from_scene(scene, "cuda")
    params = {k: v.clone().requires_grad_(True) for k, v in ds.tensors().items()}
    target = torch.from_numpy(synth.target_image(40, 40, seed=3001)).cuda()
    rgb = drk.render_autograd(params, cam, opt, sh_degree=-1)
    loss = (rgb - target).abs().mean()
    loss.backward()
    # same gradient through the plain entry points
    _, _, _, st = drk.drk_render(ds, cam, opt, need_state=True)
    dL = torch.sign(rgb.detach() - target) / rgb.numel()
    g = drk.drk_render_backward(ds, cam, opt, st, dL)
    torch.cuda.synchronize()
    # the two backward runs sum their float atomics in different orders
    for k in NAMES:
        assert params[k].grad is not None
        scale = float(g[k].abs().max())
        assert torch.allclose(params[k].grad, g[k], rtol=1e-3, atol=1e-5 * scale), k


def test_backward_paper_culling(drk):
    # the paper's lossy tile culling (Eq. 11 - Eq. 12 as printed): the
    # gradient of the image it renders, against the oracle applying the
    # same culling
    scene = synth.scene_plain(400, 8, seed=44)
    cam = synth.camera_front(48, 40)
    compare_grads(drk, scene, cam, drk.Options(cull_level=drk.CULL_PAPER), seed=45)
