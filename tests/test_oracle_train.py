"""Pins of the training oracle (supplementary "Parametrization" and "Model
Training"): closed forms of the activations, the angular-gap guarantee, the
analytic backward against central differences, Adam against torch's Adam,
and the learning-rate decay's end points."""
import math

import numpy as np
import pytest

from oracle import drk_train_oracle as T


def _raw(n, K, seed, spread=1.5, C=3):
    rng = np.random.default_rng(seed)
    return {"mu": rng.normal(size=(n, 3)), "quat": rng.normal(size=(n, 4)),
            "scale": rng.normal(-2.0, 0.5, size=(n, K)), "theta": rng.normal(0.0, spread, size=(n, K)),
            "eta": rng.normal(size=n), "tau": rng.normal(size=n), "opacity": rng.normal(size=n),
            "color": rng.normal(size=(n, C))}


def _gaps(theta):
    K = theta.shape[-1]
    nxt = np.concatenate([theta[..., 1:], theta[..., :1] + 2 * math.pi], axis=-1)
    return nxt - theta


def test_activation_closed_forms():
    raw = {"mu": np.zeros((1, 3)), "quat": np.array([[0.0, 3.0, 0.0, 4.0]]), "scale": np.log([[2.0, 0.5, 1.0]]),
           "theta": np.zeros((1, 3)), "eta": np.zeros(1), "tau": np.zeros(1), "opacity": np.zeros(1),
           "color": np.ones((1, 3))}
    a = T.activate(raw)
    np.testing.assert_allclose(a["quat"], [[0.0, 0.6, 0.0, 0.8]], atol=1e-15)
    np.testing.assert_allclose(a["scale"], [[2.0, 0.5, 1.0]], rtol=1e-15)
    # equal raw angles give equally spaced bases starting at 0
    np.testing.assert_allclose(a["theta"], [[0.0, 2 * math.pi / 3, 4 * math.pi / 3]], atol=1e-15)
    assert a["eta"][0] == 0.5 and a["opacity"][0] == 0.5
    assert a["tau"][0] == pytest.approx(-0.1 + 1.09 * 0.5, abs=1e-15)
    # tau's range is the supplement's (-0.1, 0.99)
    hi = T.activate({**raw, "tau": np.array([40.0])})["tau"][0]
    lo = T.activate({**raw, "tau": np.array([-40.0])})["tau"][0]
    assert hi == pytest.approx(0.99, abs=1e-12) and lo == pytest.approx(-0.1, abs=1e-12)
    # zero quaternion: identity rotation
    np.testing.assert_array_equal(T.activate({**raw, "quat": np.zeros((1, 4))})["quat"], [[1.0, 0, 0, 0]])


@pytest.mark.parametrize("K", [3, 4, 8, 16])
def test_theta_gaps_below_pi(K):
    # random raw angles, including saturated ones: ascending from 0, gaps sum
    # to 2 pi, every gap strictly below pi
    raw = _raw(2000, K, seed=K, spread=12.0)["theta"]
    th = T.theta_from_raw(raw)
    g = _gaps(th)
    assert np.all(th[:, 0] == 0.0)
    assert np.all(g > 0)
    np.testing.assert_allclose(g.sum(axis=1), 2 * math.pi, rtol=1e-14)
    assert g.max() < math.pi
    # the worst case (one sigmoid at its cap, the others at 0) is the bound
    # pi (1 - c / (2 - c + 2 / (K - 2))) with c = 1e-3
    x = np.full((1, K), -800.0)
    x[0, 2 % K] = 800.0
    gmax = _gaps(T.theta_from_raw(x)).max()
    c = 1e-3
    assert gmax == pytest.approx(math.pi * (1 - c / (2 - c + 2 / (K - 2))), rel=1e-12)
    # without the cap the residual 1/(K-2) puts that limit exactly at pi
    w = np.full(K, 1.0 / (K - 2))
    w[0] += 1.0
    assert 2 * math.pi * w[0] / w.sum() == pytest.approx(math.pi, rel=1e-14)


@pytest.mark.parametrize("K", [3, 8, 16])
def test_activation_backward_matches_central_differences(K):
    raw = _raw(5, K, seed=100 + K, C=12)
    rng = np.random.default_rng(200 + K)
    act = T.activate(raw)
    g = {k: rng.normal(size=np.shape(v)) for k, v in act.items()}
    an = T.activate_backward(raw, g)

    def f(r):
        a = T.activate(r)
        return sum(float(np.sum(g[k] * a[k])) for k in a)

    h = 1e-6
    for k in T.ALL:
        x = raw[k]
        num = np.zeros_like(x, dtype=np.float64)
        for idx in np.ndindex(x.shape):
            rp = {kk: np.array(vv, np.float64) for kk, vv in raw.items()}
            rm = {kk: np.array(vv, np.float64) for kk, vv in raw.items()}
            rp[k][idx] += h
            rm[k][idx] -= h
            num[idx] = (f(rp) - f(rm)) / (2 * h)
        np.testing.assert_allclose(an[k], num, rtol=1e-6, atol=1e-7, err_msg=k)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    p0 = rng.normal(size=(64,))
    grads = [rng.normal(size=(64,)) * s for s in (1.0, 0.1, 3.0, 1e-4, 1.0, 0.5)]
    for lr, eps in ((1e-2, 1e-15), (5e-3, 1e-8)):
        tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
        opt = torch.optim.Adam([tp], lr=lr, betas=(0.9, 0.999), eps=eps)
        p, m, v = p0.copy(), np.zeros(64), np.zeros(64)
        for t, g in enumerate(grads, start=1):
            tp.grad = torch.tensor(g, dtype=torch.float64)
            opt.step()
            p, m, v = T.adam(p, g, m, v, lr, t, eps=eps)
            np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_sigmoid_derivative_where_the_sigmoid_saturates():
    # sigmoid'(x) = e^-x / (1 + e^-x)^2 exactly; s (1 - s) loses it past |x| ~ 30
    for x in (30.0, 40.0, -45.0, 80.0):
        e = math.exp(-abs(x))
        assert float(T.dsigmoid(x)) == pytest.approx(e / (1 + e) ** 2, rel=1e-12)


def test_lr_exponential_end_points():
    assert T.lr_exponential(0, 5e-3, 5e-5, 35000) == pytest.approx(5e-3, rel=1e-14)
    assert T.lr_exponential(35000, 5e-3, 5e-5, 35000) == pytest.approx(5e-5, rel=1e-14)
    assert T.lr_exponential(70000, 5e-3, 5e-5, 35000) == pytest.approx(5e-5, rel=1e-14)
    # log-linear: the midpoint is the geometric mean
    assert T.lr_exponential(17500, 5e-3, 5e-5, 35000) == pytest.approx(math.sqrt(5e-3 * 5e-5), rel=1e-14)


def test_train_step_is_adam_on_the_chain_rule():
    # one fused step is the activation's chain rule (pinned above against
    # central differences) followed by Adam per array; from zero moments
    # the first Adam update is lr * sign(g)
    raw = _raw(3, 8, seed=31)
    rng = np.random.default_rng(32)
    g = {k: rng.normal(size=np.shape(v)) for k, v in T.activate(raw).items()}
    zeros = {k: np.zeros(np.shape(v)) for k, v in raw.items()}
    lr = {k: 1e-2 for k in T.ALL}
    nr, nm, nv, act = T.train_step(raw, g, zeros, zeros, lr, 1)
    g_raw = T.activate_backward(raw, g)
    for k in T.ALL:
        np.testing.assert_allclose(nr[k], raw[k] - lr[k] * np.sign(g_raw[k]), rtol=0, atol=1e-12)
        np.testing.assert_allclose(nm[k], 0.1 * g_raw[k], rtol=1e-14)
        np.testing.assert_allclose(nv[k], 0.001 * g_raw[k] ** 2, rtol=1e-14)
    np.testing.assert_allclose(act["opacity"], 1 / (1 + np.exp(-nr["opacity"])), rtol=1e-15)
