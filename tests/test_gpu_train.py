"""GPU tests of the training path (supplementary "Parametrization" and
"Model Training"): the activation kernel, its backward and the fused Adam
step against the FP64 training oracle, argument checks, and a short fit of a
synthetic shape image through the renderer, its backward and the optimiser."""
import numpy as np
import pytest

from oracle import drk_train_oracle as T
from paper_2412_11752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ("mu", "quat", "scale", "theta", "eta", "tau", "opacity", "color")


@pytest.fixture(scope="module")
def drk():
    from paper_2412_11752_gb300 import drk as D
    D.lib()
    return D


def _raw_arrays(n, K, seed, sh_degree=-1, spread=2.0):
    rng = np.random.default_rng(seed)
    C = 3 if sh_degree < 0 else 3 * (sh_degree + 1) ** 2
    a = {"mu": rng.normal(size=(n, 3)), "quat": rng.normal(size=(n, 4)),
         "scale": rng.normal(-2.0, 1.0, size=(n, K)), "theta": rng.normal(0.0, spread, size=(n, K)),
         "eta": rng.normal(0, spread, size=n), "tau": rng.normal(0, spread, size=n),
         "opacity": rng.normal(0, spread, size=n), "color": rng.normal(size=(n, C // 3, 3) if sh_degree >= 0 else (n, 3))}
    # saturated values and a zero quaternion
    a["theta"][:3] = np.array([40.0, -40.0, 12.0] * K)[: 3 * K].reshape(3, K)
    a["opacity"][0], a["tau"][1], a["eta"][2] = 30.0, -30.0, 18.0
    a["quat"][4] = 0.0
    return {k: np.ascontiguousarray(v, np.float32) for k, v in a.items()}


def _to_np(d):
    return {k: d[k].detach().cpu().numpy().astype(np.float64) for k in NAMES if d.get(k) is not None}


def _close(got, want, rtol, atol, what):
    err = np.abs(got - want)
    bound = atol + rtol * np.abs(want)
    bad = err > bound
    assert not bad.any(), f"{what}: {bad.sum()} of {bad.size} off, max err {err.max():.3e} at {np.argmax(err)}"


@pytest.mark.parametrize("K,sh", [(3, -1), (8, -1), (12, 1), (16, 3)])
def test_activate_matches_oracle(drk, K, sh):
    a = _raw_arrays(3000, K, seed=700 + K, sh_degree=sh)
    raw = drk.RawScene.from_arrays(a, sh_degree=sh)
    act = drk.activate(raw)
    torch.cuda.synchronize()
    ref = T.activate({k: a[k].astype(np.float64) for k in NAMES})
    got = _to_np(act.tensors())
    for k in T.ACTIVATED:
        _close(got[k], ref[k], 2e-6, 4e-6 if k == "theta" else 1e-6, k)
    assert act.mu.data_ptr() == raw.mu.data_ptr() and act.color.data_ptr() == raw.color.data_ptr()
    # every angular gap below pi in float32 too
    th = got["theta"]
    gaps = np.diff(np.concatenate([th, th[:, :1] + 2 * np.pi], axis=1), axis=1)
    assert gaps.min() > 0 and gaps.max() < np.pi


@pytest.mark.parametrize("K", [3, 8, 16])
def test_activate_backward_matches_oracle(drk, K):
    a = _raw_arrays(2000, K, seed=800 + K)
    rng = np.random.default_rng(900 + K)
    g = {k: np.ascontiguousarray(rng.normal(size=v.shape), np.float32) for k, v in a.items()}
    raw = drk.RawScene.from_arrays(a)
    g_dev = {k: torch.from_numpy(v).cuda() for k, v in g.items()}
    got = _to_np(drk.activate_backward(raw, g_dev))
    torch.cuda.synchronize()
    ref = T.activate_backward({k: v.astype(np.float64) for k, v in a.items()},
                              {k: v.astype(np.float64) for k, v in g.items()})
    for k in NAMES:
        scale = np.abs(ref[k]).max() + 1e-30
        _close(got[k], ref[k], 1e-5, 1e-6 * scale, k)


@pytest.mark.parametrize("K,sh", [(8, -1), (16, 2)])
def test_adam_steps_match_oracle(drk, K, sh):
    a = _raw_arrays(2500, K, seed=1000 + K, sh_degree=sh, spread=1.0)
    raw = drk.RawScene.from_arrays(a, sh_degree=sh)
    opt = drk.Adam(raw)
    r = {k: v.astype(np.float64) for k, v in a.items()}
    m = {k: np.zeros_like(v) for k, v in r.items()}
    v = {k: np.zeros_like(x) for k, x in r.items()}
    rng = np.random.default_rng(1100 + K)
    for t in range(1, 4):
        lr = {k: float(x) for k, x in zip(NAMES, (2e-3, 1e-3, 5e-3, 5e-3, 4e-3, 3e-3, 5e-2, 2.5e-3))}
        g = {k: np.ascontiguousarray(rng.normal(size=x.shape) * (1.0 + t), np.float32) for k, x in a.items()}
        scene = opt.step({k: torch.from_numpy(x).cuda() for k, x in g.items()}, lr)
        torch.cuda.synchronize()
        # the oracle takes the float32 values of the hyper-parameters the GPU uses
        lr32 = {k: float(np.float32(x)) for k, x in lr.items()}
        r, m, v, act = T.train_step(r, {k: x.astype(np.float64) for k, x in g.items()}, m, v, lr32, t,
                                    beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)),
                                    eps=float(np.float32(1e-15)))
        got_raw, got_m, got_v = _to_np(raw.tensors()), _to_np(opt.m), _to_np(opt.v)
        got_act = _to_np(scene.tensors())
        for k in NAMES:
            _close(got_raw[k], r[k], 1e-6, 2e-6, f"raw {k} step {t}")
            _close(got_m[k], m[k], 1e-5, 1e-6 * np.abs(m[k]).max(), f"m {k} step {t}")
            _close(got_v[k], v[k], 1e-5, 1e-6 * np.abs(v[k]).max(), f"v {k} step {t}")
        for k in T.ACTIVATED:
            _close(got_act[k], act[k], 1e-5, 1e-5, f"activated {k} step {t}")
        # continue from the float32 state, as the GPU does
        r = {k: x.astype(np.float32).astype(np.float64) for k, x in _to_np(raw.tensors()).items()}


def test_training_argument_errors(drk):
    a = _raw_arrays(10, 8, seed=5)
    raw = drk.RawScene.from_arrays(a)
    opt = drk.Adam(raw)
    g = {k: torch.zeros_like(x) for k, x in raw.tensors().items()}
    lr = drk.learning_rates(0)
    opt.t = -1                      # next step would be t = 0
    with pytest.raises(drk.DrkError) as e:
        opt.step(g, lr)
    assert e.value.code == 1
    opt.t = 0
    bad = dict(lr, mu=float("nan"))
    with pytest.raises(drk.DrkError) as e:
        opt.step(g, bad)
    assert e.value.code == 1
    raw2 = drk.RawScene.from_arrays({**a, "scale": a["scale"][:, :2], "theta": a["theta"][:, :2]})
    with pytest.raises(drk.DrkError) as e:
        drk.activate(raw2)
    assert e.value.code == 1
    # empty scene: nothing launched, no error
    empty = drk.RawScene.from_arrays({k: v[:0] for k, v in a.items()})
    drk.activate(empty)


def test_fit_shape_target(drk):
    # a few hundred DRKs fitted to a synthetic image of convex shapes: the L1
    # loss falls to a quarter of its start through render -> backward ->
    # fused Adam
    H = W = 64
    cam = synth.camera_front(W, H)
    target = torch.from_numpy(synth.shape_target(H, W)).cuda()
    raw = drk.RawScene.from_arrays(synth.raw_scene(400, 8, seed=6001))
    opt = drk.Adam(raw)
    ropt = drk.Options(bg=(0.35, 0.35, 0.35))
    sched = dict(drk.LR_SCHEDULE, mu=(2e-3, 2e-4), color=(1e-2, 1e-3))
    losses = []
    for step in range(200):
        rgb, _, _, st = drk.drk_render(opt.scene, cam, ropt, need_state=True)
        diff = rgb - target
        losses.append(float(diff.abs().mean()))
        dL = torch.sign(diff) / diff.numel()
        g = drk.drk_render_backward(opt.scene, cam, ropt, st, dL)
        st.free()
        opt.step(g, drk.learning_rates(step, 200, sched))
    torch.cuda.synchronize()
    assert all(np.isfinite(losses))
    first, last = np.mean(losses[:5]), np.mean(losses[-5:])
    print(f"L1 loss {first:.4f} -> {last:.4f} (ratio {last / first:.3f})")
    assert last < 0.25 * first, (first, last)          # measured: 0.142 -> 0.012
    th = opt.scene.theta.cpu().numpy()
    gaps = np.diff(np.concatenate([th, th[:, :1] + 2 * np.pi], axis=1), axis=1)
    assert gaps.max() < np.pi and gaps.min() > 0
