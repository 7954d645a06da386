"""Sorting-accuracy study of the cache-sorting order (supplementary
"Cache-Sorting" paragraph and its figure on sorting accuracy): DRKs sampled
at random in a volume, the per-pixel order in which a tile's pairs are
processed under several pre-sort keys, with and without a sorted cache,
compared with the exact r_t order by accuracy, Kendall's tau and MAE.

Readings (the paper names the metrics and pre-sort keys but not their
definitions):
  * the exact order of a pixel is its contributors (alpha_tilde >= alpha_min)
    sorted by (r_t, index), r_t of Eq. 13 as the oracle computes it;
  * pre-sort keys, one value per (tile, primitive), ties by index:
      random   - a seeded random permutation ("cache-sorting alone"),
      centre   - view depth of the centre mu (the 3D-GS order),
      nearest  - the smallest r_t of the primitive over the tile's pixels it
                 contributes to (nearest distance between DRK and tile),
      centric  - r_t on the ray through the tile point nearest to the
                 projected centre of mu (the "most centric" point);
  * the cache holds up to `cache` entries sorted by (r_t, index) and, when a
    new entry overfills it, processes its smallest (the oracle's reading of
    Sec. 4.4); cache 0 processes the pre-sort order as it is;
  * accuracy = share of positions where the processed primitive is the
    exact one; Kendall's tau between processed and exact positions, averaged
    over pixels with at least two contributors; MAE = mean |r_t processed -
    r_t exact| over positions.

Run as a script to print the table:  python tests/sort_study.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import drk_oracle as O  # noqa: E402
from paper_2412_11752_gb300 import synth  # noqa: E402

TILE = 16
KEYS = ("random", "centre", "nearest", "centric")


def kendall_tau(order: np.ndarray) -> float:
    """Kendall's tau between positions 0..n-1 and `order` (a permutation of
    the exact ranks): (concordant - discordant) / (n (n - 1) / 2)."""
    o = np.asarray(order)
    n = len(o)
    if n < 2:
        return 1.0
    s = 0
    for i in range(n - 1):
        s += int(np.sum(np.sign(o[i + 1:] - o[i])))
    return s / (n * (n - 1) / 2)


def cache_process(ranks_in_arrival: list[int], cache: int) -> list[int]:
    """Processing order of exact ranks met in arrival order, through a cache
    kept sorted that processes its smallest entry when overfilled."""
    if cache <= 0:
        return list(ranks_in_arrival)
    buf: list[int] = []
    out: list[int] = []
    for r in ranks_in_arrival:
        j = len(buf)
        buf.append(r)
        while j > 0 and buf[j - 1] > r:
            buf[j] = buf[j - 1]
            j -= 1
        buf[j] = r
        if len(buf) > cache:
            out.append(buf.pop(0))
    return out + buf


def _ray_world(cam, x: float, y: float) -> np.ndarray:
    """World direction of the camera ray through image point (x, y), scaled
    so that its view-space z is 1 (r_t along it is the view depth)."""
    M = np.asarray(cam.world_to_cam, np.float64)
    dc = np.array([(x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0])
    return M[:, :3].T @ dc


def _cam_centre(cam) -> np.ndarray:
    M = np.asarray(cam.world_to_cam, np.float64)
    return -M[:, :3].T @ M[:, 3]


def tile_lists(scene, cam, opt, tx: int, ty: int):
    """Exact contributor lists (idx, r_t) of the pixels of one tile."""
    out = []
    for y in range(ty * TILE, min((ty + 1) * TILE, cam.height)):
        for x in range(tx * TILE, min((tx + 1) * TILE, cam.width)):
            idx, t, _, _ = O.contributors(scene, cam, opt, x, y)
            out.append((np.asarray(idx), np.asarray(t)))
    return out


def presort_keys(scene, cam, lists, tx: int, ty: int, rng) -> dict[str, dict[int, float]]:
    prims = sorted({int(i) for idx, _ in lists for i in idx})
    M = np.asarray(cam.world_to_cam, np.float64)
    mu = np.asarray(scene.mu, np.float64)
    o = _cam_centre(cam)
    keys = {k: {} for k in KEYS}
    perm = rng.permutation(len(prims))
    near: dict[int, float] = {}
    for idx, t in lists:
        for i, ti in zip(idx, t):
            near[int(i)] = min(near.get(int(i), np.inf), float(ti))
    x0, y0 = tx * TILE + 0.5, ty * TILE + 0.5
    x1 = min((tx + 1) * TILE, cam.width) - 0.5
    y1 = min((ty + 1) * TILE, cam.height) - 0.5
    for j, i in enumerate(prims):
        keys["random"][i] = float(perm[j])
        pc = M[:, :3] @ mu[i] + M[:, 3]
        keys["centre"][i] = float(pc[2])
        keys["nearest"][i] = near[i]
        # projected centre clamped into the tile (behind the camera: tile centre)
        if pc[2] > 0:
            u = cam.fx * pc[0] / pc[2] + cam.cx
            v = cam.fy * pc[1] / pc[2] + cam.cy
        else:
            u, v = 0.5 * (x0 + x1), 0.5 * (y0 + y1)
        u, v = min(max(u, x0), x1), min(max(v, y0), y1)
        Rz = O.rotation(scene.quat[i])[:, 2]
        d = _ray_world(cam, u, v)
        dn = float(d @ Rz)
        keys["centric"][i] = float((mu[i] - o) @ Rz / dn) if abs(dn) > 1e-12 else np.inf
    return keys


def pixel_metrics(idx: np.ndarray, t: np.ndarray, key: dict[int, float], cache: int):
    """(hits, positions, tau, abs depth error sum) of one pixel."""
    n = len(idx)
    arrival = sorted(range(n), key=lambda r: (key[int(idx[r])], int(idx[r])))
    proc = np.asarray(cache_process(arrival, cache))
    hits = int(np.sum(proc == np.arange(n)))
    return hits, n, kendall_tau(proc), float(np.sum(np.abs(t[proc] - t)))


def study(n: int = 1500, seed: int = 5150, width: int = 64, height: int = 64, caches=(0, 8),
          tiles=None) -> dict:
    """Metrics per (pre-sort key, cache length) over the tiles of one random
    scene: {(key, cache): {"accuracy", "tau", "mae", "pixels", "positions"}}."""
    scene = synth.scene_plain(n, 8, seed=seed)
    cam = synth.camera_front(width, height)
    opt = O.Options()
    rng = np.random.default_rng(seed + 1)
    if tiles is None:
        tiles = [(tx, ty) for ty in range((height + TILE - 1) // TILE) for tx in range((width + TILE - 1) // TILE)]
    acc = {(k, c): [0, 0, 0.0, 0, 0.0] for k in KEYS for c in caches}
    for tx, ty in tiles:
        lists = tile_lists(scene, cam, opt, tx, ty)
        keys = presort_keys(scene, cam, lists, tx, ty, rng)
        for idx, t in lists:
            if len(idx) < 2:
                continue
            for k in KEYS:
                for c in caches:
                    h, m, tau, err = pixel_metrics(idx, t, keys[k], c)
                    a = acc[(k, c)]
                    a[0] += h
                    a[1] += m
                    a[2] += tau
                    a[3] += 1
                    a[4] += err
    return {kc: {"accuracy": a[0] / max(1, a[1]), "tau": a[2] / max(1, a[3]), "mae": a[4] / max(1, a[1]),
                 "pixels": a[3], "positions": a[1]} for kc, a in acc.items()}


def main():
    res = study()
    print(f"{'pre-sort':10s} {'cache':>5s} {'accuracy':>9s} {'tau':>7s} {'MAE':>9s}")
    for (k, c), r in res.items():
        print(f"{k:10s} {c:5d} {r['accuracy']:9.4f} {r['tau']:7.4f} {r['mae']:9.5f}")
    any_r = next(iter(res.values()))
    print(f"pixels {any_r['pixels']}, positions {any_r['positions']}")


if __name__ == "__main__":
    main()
