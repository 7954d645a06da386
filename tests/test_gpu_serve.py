"""GPU tests of the serving loop (drk_serve_*): a batched image is the image
drk_render gives for the same scene and camera, bit for bit, whatever the
batch it was rendered in; budget, timeout, release and injected allocation
failures complete with their documented status and leave the server usable."""
import numpy as np
import pytest

from paper_2412_11752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OOM, TIMEOUT, BUSY, NOT_FOUND, INVALID = 2, 5, 6, 7, 1


@pytest.fixture(scope="module")
def drk():
    from paper_2412_11752_gb300 import drk as D
    D.lib()
    return D


@pytest.fixture(scope="module")
def scenes(drk):
    hs = [synth.scene_clustered(6000, 8, seed=4101), synth.scene_plain(2500, 5, seed=4102),
          synth.scene_clustered(12000, 8, seed=4103, sh_degree=1),
          synth.scene_plain(1500, 12, seed=4104)]            # K = 12: the 16-basis class
    return hs, [drk.DeviceScene.from_scene(s, "cuda") for s in hs]


def _requests(count, seed, n_scenes):
    rng = np.random.default_rng(seed)
    sizes = [(96, 64), (160, 120), (200, 150), (64, 64), (250, 100)]
    out = []
    for _ in range(count):
        w, h = sizes[int(rng.integers(0, len(sizes)))]
        out.append((int(rng.integers(0, n_scenes)), synth.camera_on_sphere(rng, w, h)))
    return out


def _reference(drk, dscene, cam, opt):
    rgb, _, _, _ = drk.drk_render(dscene, cam, opt)
    torch.cuda.synchronize()
    return rgb.clone()


@pytest.mark.parametrize("max_batch", [1, 8, 64])
def test_batched_images_equal_single_renders(drk, scenes, max_batch):
    _, ds = scenes
    opt = drk.Options()
    reqs = _requests(24, seed=77, n_scenes=len(ds))
    with drk.Server(0, mem_budget=4 << 30, max_batch=max_batch, opt=opt) as srv:
        ids = [srv.add_scene(d) for d in ds]
        outs, tickets = [], []
        for sid, cam in reqs:
            o = torch.full((3, cam.height, cam.width), float("nan"), device="cuda")
            outs.append(o)
            tickets.append(srv.submit(ids[sid], cam, o))
        timings = [srv.wait(t, 60000) for t in tickets]
    for (sid, cam), o, t in zip(reqs, outs, timings):
        assert t["status"] == 0
        assert t["arrival_ms"] <= t["start_ms"] <= t["end_ms"]
        assert 1 <= t["batch_size"] <= max_batch
        ref = _reference(drk, ds[sid], cam, opt)
        assert torch.equal(o, ref), f"scene {sid} {cam.width}x{cam.height}"
    if max_batch > 1:
        assert max(t["batch_size"] for t in timings) > 1   # requests were really batched


def test_requests_while_running_and_release(drk, scenes):
    _, ds = scenes
    opt = drk.Options()
    reqs = _requests(12, seed=91, n_scenes=len(ds))
    with drk.Server(0, mem_budget=4 << 30, max_batch=4, opt=opt) as srv:
        ids = [srv.add_scene(d) for d in ds]
        pending = []
        for k, (sid, cam) in enumerate(reqs):
            o = torch.zeros((3, cam.height, cam.width), device="cuda")
            pending.append((srv.submit(ids[sid], cam, o), sid, cam, o))
            if k % 3 == 2:                  # let the worker pick up what is queued
                srv.wait(pending[-1][0], 60000)
        for tk, sid, cam, o in pending:
            t = srv.wait(tk, 60000)
            assert t["status"] == 0
            assert torch.equal(o, _reference(drk, ds[sid], cam, opt))
            done, _ = srv.poll(tk)
            assert done
            srv.release(tk)
            with pytest.raises(drk.DrkError) as e:
                srv.poll(tk)
            assert e.value.code == NOT_FOUND


def test_over_budget_request_fails_and_server_continues(drk, scenes):
    _, ds = scenes
    opt = drk.Options()
    with drk.Server(0, mem_budget=6 << 20, max_batch=4, opt=opt) as srv:
        sid = srv.add_scene(ds[1])
        big = synth.camera_front(3840, 2160)
        o_big = torch.zeros((3, 2160, 3840), device="cuda")
        t_big = srv.wait(srv.submit(sid, big, o_big), 60000)
        assert t_big["status"] == OOM
        small = synth.camera_front(96, 64)
        o = torch.zeros((3, 64, 96), device="cuda")
        t = srv.wait(srv.submit(sid, small, o), 60000)
        assert t["status"] == 0
        assert torch.equal(o, _reference(drk, ds[1], small, opt))


def test_injected_allocation_failure(drk, scenes):
    _, ds = scenes
    opt = drk.Options()
    cam = synth.camera_front(160, 120)
    with drk.Server(0, mem_budget=4 << 30, max_batch=1, opt=opt) as srv:
        sid = srv.add_scene(ds[0])
        for n in (0, 3, 9, 17):             # phase A (early, late), phase B, batch tile order
            srv.inject_alloc_failure(n)
            o = torch.zeros((3, 120, 160), device="cuda")
            t = srv.wait(srv.submit(sid, cam, o), 60000)
            assert t["status"] == OOM, n
        srv.inject_alloc_failure(-1)
        o = torch.zeros((3, 120, 160), device="cuda")
        t = srv.wait(srv.submit(sid, cam, o), 60000)
        assert t["status"] == 0
        assert torch.equal(o, _reference(drk, ds[0], cam, opt))


def test_wait_timeout_and_argument_errors(drk):
    opt = drk.Options()
    big = synth.scene_clustered(100_000, 8, seed=2000)
    dbig = drk.DeviceScene.from_scene(big, "cuda")
    with drk.Server(0, mem_budget=8 << 30, max_batch=2, opt=opt) as srv:
        sid = srv.add_scene(dbig)
        cam = synth.camera_front(1920, 1080)
        o = torch.zeros((3, 1080, 1920), device="cuda")
        tk = srv.submit(sid, cam, o)
        with pytest.raises(drk.DrkError) as e:
            srv.wait(tk, 0.0)           # a 1080p frame of 100k primitives is not done at once
        assert e.value.code == TIMEOUT
        try:
            srv.release(tk)             # refused while the ticket is not done
            released = True
        except drk.DrkError as err:
            assert err.code == BUSY
            released = False
        if not released:
            assert srv.wait(tk, 60000)["status"] == 0
            srv.release(tk)
        with pytest.raises(drk.DrkError) as e:
            srv.submit(99, cam, o)
        assert e.value.code == NOT_FOUND
        bad = synth.camera_front(8, 8)
        bad.fx = -1.0
        with pytest.raises(drk.DrkError) as e:
            srv.submit(sid, bad, torch.zeros((3, 8, 8), device="cuda"))
        assert e.value.code == INVALID


def test_served_images_match_the_oracle_at_serving_resolutions(drk):
    # a mixed batch of 640 x 480 and 3840 x 2160 requests (and one 1280 x
    # 720) over two resident scenes, rendered by the batch raster; sampled
    # pixels plus two whole tiles of every request against the FP64 oracle
    from helpers import image_parity, oracle_options
    from oracle import drk_oracle as O
    hs = [synth.scene_clustered(20000, 8, seed=4201), synth.scene_clustered(20000, 8, seed=4202, n_clusters=40)]
    ds = [drk.DeviceScene.from_scene(s, "cuda") for s in hs]
    rng = np.random.default_rng(4203)
    reqs = [(i % 2, synth.camera_on_sphere(rng, *wh))
            for i, wh in enumerate([(640, 480), (3840, 2160), (640, 480), (3840, 2160), (1280, 720)])]
    opt = drk.Options()
    with drk.Server(0, mem_budget=16 << 30, max_batch=8, opt=opt) as srv:
        ids = [srv.add_scene(d) for d in ds]
        outs = [torch.full((3, c.height, c.width), float("nan"), device="cuda") for _, c in reqs]
        tickets = [srv.submit(ids[sid], cam, o) for (sid, cam), o in zip(reqs, outs)]
        timings = [srv.wait(t, 120000) for t in tickets]
    assert max(t["batch_size"] for t in timings) > 1
    for k, ((sid, cam), o, t) in enumerate(zip(reqs, outs, timings)):
        assert t["status"] == 0
        tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
        pix = synth.pixel_sample(cam.width, cam.height, 512, seed=4300 + k, tiles=[(tx // 2, ty // 2), (tx - 1, ty - 1)])
        ref = O.render_pixels(hs[sid], cam, oracle_options(opt), pix)
        img = o.cpu().numpy()
        image_parity(img[:, pix[:, 1], pix[:, 0]], ref, 2, f"served {cam.width}x{cam.height}")


def test_batch_device_timeline(drk, scenes):
    # every request reports its batch's device timeline: phase A, phase B
    # and the raster in order, on one of the two server streams
    _, ds = scenes
    reqs = _requests(16, seed=79, n_scenes=len(ds))
    with drk.Server(0, mem_budget=4 << 30, max_batch=4) as srv:
        ids = [srv.add_scene(d) for d in ds]
        outs = [torch.empty((3, c.height, c.width), device="cuda") for _, c in reqs]
        tickets = [srv.submit(ids[sid], cam, o) for (sid, cam), o in zip(reqs, outs)]
        for t in tickets:
            srv.wait(t, 60000)
        tl = [srv.timeline(t, 60000) for t in tickets]
    for t in tl:
        assert t["status"] == 0 and t["stream"] in (0, 1)
        assert 0.0 < t["dev_a0_ms"] <= t["dev_a1_ms"] <= t["dev_b1_ms"] <= t["dev_r1_ms"]
