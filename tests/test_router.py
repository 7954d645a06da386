"""Request-level serving replicas (Router): the least-loaded routing policy
with stand-in servers on the CPU, and, on a GPU, two servers on one device
whose images equal drk_render's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2412_11752_gb300 import drk, synth  # noqa: E402


class FakeServer:
    """Stands in for drk.Server: tickets finish when the test says so."""

    def __init__(self, dev):
        self.dev = dev
        self.done = set()
        self.submitted = []
        self.n = 0

    def add_scene(self, ds):
        return 0

    def submit(self, sid, cam, img):
        self.n += 1
        self.submitted.append((cam.width, cam.height))
        return self.n

    def poll(self, tk):
        return tk in self.done, {}

    def wait(self, tk, timeout_ms=0):
        self.done.add(tk)
        return {"status": 0}

    def release(self, tk):
        pass

    def close(self):
        pass


class HostScene:
    def __init__(self, n):
        self.mu = np.zeros((n, 3), np.float32)


def test_least_loaded_policy():
    assert drk.least_loaded([3.0, 1.0, 1.0, 2.0]) == 1
    assert drk.least_loaded([0.0]) == 0
    assert drk.least_loaded([5.0, 5.0]) == 0


def test_router_routes_to_the_least_loaded_server(monkeypatch):
    # images are allocated on the server's device; keep them on the CPU here
    monkeypatch.setattr(drk.torch, "empty", lambda *a, **k: None)
    r = drk.Router([0, 1, 2], make_server=FakeServer)
    r.scene_ids.append([0, 0, 0])
    r.scene_n.append(100)
    cams = [synth.camera_front(w, h) for w, h in ((400, 300), (100, 100), (100, 100), (200, 100), (50, 50))]
    tk = [r.submit(0, c) for c in cams]
    # 400x300 -> s0; 100x100 -> s1; 100x100 -> s2; 200x100 -> s1 (1e6 < 1.2e7),
    # then s2 (1e6) is least loaded
    assert [r.server_of(t) for t in tk] == [0, 1, 2, 1, 2]
    assert r.load == [400 * 300 * 100, (100 * 100 + 200 * 100) * 100, (100 * 100 + 50 * 50) * 100]
    # finishing server 0's request frees it for the next one
    r.wait(tk[0])
    assert r.load[0] == 0
    nxt = r.submit(0, synth.camera_front(64, 64))
    assert r.server_of(nxt) == 0
    # a request another caller finished is reaped at the next submit
    r.servers[1].done.update({1, 2})
    last = r.submit(0, synth.camera_front(8, 8))
    assert r.server_of(last) == 1 and r.load[1] == 8 * 8 * 100


@pytest.mark.gpu
def test_two_replicas_on_one_gpu_give_drk_render_images():
    drk.lib()
    hs = [synth.scene_clustered(5000, 8, seed=4401), synth.scene_plain(2000, 8, seed=4402)]
    rng = np.random.default_rng(4403)
    reqs = [(i % 2, synth.camera_on_sphere(rng, *wh))
            for i, wh in enumerate([(160, 120), (96, 64), (200, 150), (64, 64), (160, 120), (250, 100)] * 2)]
    opt = drk.Options()
    with drk.Router([0, 0], mem_budget=4 << 30, max_batch=4, opt=opt) as r:
        ids = [r.add_scene(s) for s in hs]
        tickets = [r.submit(ids[sid], cam) for sid, cam in reqs]
        used = {r.server_of(t) for t in tickets}
        timings = [r.wait(t, 60000) for t in tickets]
        imgs = [r.image(t).clone() for t in tickets]
    assert used == {0, 1}
    for (sid, cam), t, img in zip(reqs, timings, imgs):
        assert t["status"] == 0
        ref, _, _, _ = drk.drk_render(drk.DeviceScene.from_scene(hs[sid], "cuda"), cam, opt)
        torch.cuda.synchronize()
        assert torch.equal(img, ref)
