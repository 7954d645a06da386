"""The sorting-accuracy study (supplementary "Cache-Sorting" paragraph): its
metrics against library and brute-force definitions, its cache against the
oracle's cache-sorting order, and the paper's findings on random DRKs."""
import itertools

import numpy as np
import pytest

import sort_study as S
from oracle import drk_oracle as O
from paper_2412_11752_gb300 import synth


def test_kendall_tau_matches_scipy():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(11)
    for n in (2, 3, 7, 40):
        for _ in range(5):
            p = rng.permutation(n)
            assert S.kendall_tau(p) == pytest.approx(stats.kendalltau(np.arange(n), p).statistic, abs=1e-12)
    assert S.kendall_tau(np.arange(9)) == 1.0
    assert S.kendall_tau(np.arange(9)[::-1]) == -1.0


def test_cache_process_brute_force():
    # cache 0: the arrival order; a cache at least as long as the list: sorted
    rng = np.random.default_rng(12)
    for n in (1, 5, 12):
        a = list(rng.permutation(n))
        assert S.cache_process(a, 0) == a
        assert S.cache_process(a, n) == sorted(a)
    # a cache of c entries processes, at each arrival past the c-th, the
    # smallest of what has arrived and is not processed yet
    for a in itertools.permutations(range(6)):
        for c in (1, 2, 3):
            out, seen = [], []
            for k, r in enumerate(a):
                seen.append(r)
                if k >= c:
                    m = min(seen)
                    seen.remove(m)
                    out.append(m)
            assert S.cache_process(list(a), c) == out + sorted(seen)


def test_cache_matches_oracle_cache_sorting_order():
    # the study's cache with the centre-depth key is the oracle's order_mode 1
    scene = synth.scene_plain(600, 8, seed=5101)
    cam = synth.camera_front(32, 32)
    exact_opt = O.Options()
    lit_opt = O.Options(order_mode=1, cache_len=8)
    M = np.asarray(cam.world_to_cam, np.float64)
    zc = M[2, :3] @ np.asarray(scene.mu, np.float64).T + M[2, 3]
    checked = 0
    for x, y in ((3, 4), (16, 16), (20, 9), (30, 28)):
        idx, t, _, _ = O.contributors(scene, cam, exact_opt, x, y)
        lidx, _, _, _ = O.contributors(scene, cam, lit_opt, x, y)
        key = {int(i): float(zc[int(i)]) for i in idx}
        arrival = sorted(range(len(idx)), key=lambda r: (key[int(idx[r])], int(idx[r])))
        proc = S.cache_process(arrival, 8)
        np.testing.assert_array_equal(np.asarray(idx)[proc], lidx)
        checked += len(idx) > 8
    assert checked >= 2     # some pixels overflow the cache


def test_study_reproduces_the_papers_findings():
    r = S.study(n=900, seed=5152, width=48, height=48, caches=(0, 8))
    for k in S.KEYS:       # the cache corrects most disorders of every pre-sort
        assert r[(k, 8)]["accuracy"] > r[(k, 0)]["accuracy"]
        assert r[(k, 8)]["tau"] > r[(k, 0)]["tau"]
        assert r[(k, 8)]["mae"] < r[(k, 0)]["mae"]
    # nearest distance between DRK and tile is the best pre-sort; it and the
    # most centric one beat the centre-depth (3D-GS) pre-sort, and every
    # pre-sort beats cache-sorting alone
    acc = {k: r[(k, 8)]["accuracy"] for k in S.KEYS}
    assert acc["nearest"] == max(acc.values())
    assert acc["nearest"] > acc["centre"] and acc["centric"] > acc["centre"]
    assert min(acc["centre"], acc["centric"], acc["nearest"]) > acc["random"]
    assert r[("nearest", 8)]["tau"] > 0.99
