"""GPU reverse mode against the oracle's analytic (back-to-front) derivative.

The oracle's derivative is itself pinned to FP64 central differences
(test_oracle_pins.py); here the CUDA backward, which replays the forward
front to back, must agree with it per parameter tensor."""
import numpy as np
import pytest

from helpers import TOL_GRAD_REL, excluded, oracle_options, rel_err
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
    w[:, excluded(ref_f["flags"])] = 0.0           # drop threshold-decided pixels
    g = drk.drk_render_backward(ds, cam, opt, st, torch.from_numpy(w.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    st.free()
    ref = O.render_backward(scene, cam, oopt, w)
    report = {}
    for k in names:
        a = g[k].cpu().numpy().astype(np.float64)
        b = ref[k]
        r = rel_err(a, b)
        report[k] = r
        assert np.all(np.isfinite(a)), k
        assert r <= tol, f"{k}: relative error {r:.2e} (all: {report})"
        bound = 1e-3 * np.abs(b).max() + 1e-3 * np.abs(b) + 1e-7
        worst = np.max(np.abs(a - b) - bound)
        assert worst <= 0, f"{k}: elementwise excess {worst:.2e}"
    return report


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
