"""Seeded synthetic DRK scenes, cameras and targets.

This module only draws random inputs: it holds none of the method's
arithmetic (no projection, no kernel evaluation, no compositing).  Both the
CUDA path and the FP64 oracle are fed from here, so that they see the same
float32 values.

Primitive parameters follow the activated parametrisation of Sec. 4 (mu, q,
s_k, theta_k, eta, tau, o, colour) and the ranges of the supplementary
"Parametrization" paragraph: o in (0, 1), s_k > 0, tau in (-0.1, 0.99),
eta in (0, 1), K ascending polar angles.  The generator rejects angle sets
whose largest cyclic gap exceeds pi - 0.05, so that every sector of Eq. 7 is
well conditioned (the activation of the supplement keeps gaps below pi).

Scene families (sizes and distributions of the paper's workloads, which the
paper measures on DiverseScenes with 42K-260K primitives and K = 8):

* ``scene_plain``      -- uniform centres in the unit cube, plain RGB.
* ``scene_clustered``  -- planar surface clusters plus a uniform background,
                          degree-3 SH colour (48 coefficients).
* ``scene_slab``       -- heavy depth overlap: all centres in a 0.5-unit slab,
                          near-hard edges (tau close to its upper end).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

SH_DC_SCALE = 1.0 / (2.0 * math.sqrt(math.pi))   # value of the l = 0 real SH
TWO_PI = 2.0 * math.pi
MAX_GAP = math.pi - 0.05


@dataclass
class Scene:
    """Activated DRK parameters, float32, structure of arrays."""
    mu: np.ndarray          # (n, 3)
    quat: np.ndarray        # (n, 4) w, x, y, z (not necessarily unit)
    scale: np.ndarray       # (n, K) > 0
    theta: np.ndarray       # (n, K) ascending, span < 2 pi
    eta: np.ndarray         # (n,)
    tau: np.ndarray         # (n,)
    opacity: np.ndarray     # (n,)
    color: np.ndarray       # (n, 3) plain RGB or (n, (deg+1)^2, 3) SH
    sh_degree: int = -1     # -1 = plain RGB

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    @property
    def K(self) -> int:
        return int(self.scale.shape[1])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.mu[idx], self.quat[idx], self.scale[idx], self.theta[idx],
                     self.eta[idx], self.tau[idx], self.opacity[idx], self.color[idx],
                     self.sh_degree)

    def arrays(self) -> dict:
        return dict(mu=self.mu, quat=self.quat, scale=self.scale, theta=self.theta,
                    eta=self.eta, tau=self.tau, opacity=self.opacity, color=self.color)

    def copy(self) -> "Scene":
        return Scene(**{k: v.copy() for k, v in self.arrays().items()},
                     sh_degree=self.sh_degree)


@dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    ``world_to_cam`` is the 3x4 row-major [R | t] with x_cam = R x_world + t.
    Pixel (x, y) has its centre at (x + 0.5, y + 0.5).
    """
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    world_to_cam: np.ndarray = field(default_factory=lambda: np.eye(3, 4, dtype=np.float32))

    @property
    def npix(self) -> int:
        return self.width * self.height


# --------------------------------------------------------------------------
# cameras

def _focal(height: int, fov_y_deg: float) -> float:
    return height / (2.0 * math.tan(math.radians(fov_y_deg) / 2.0))


def camera_lookat(width: int, height: int, eye, target, fov_y_deg: float = 50.0,
                  down_hint=(0.0, 1.0, 0.0)) -> Camera:
    """Camera at ``eye`` looking at ``target``; image-down follows ``down_hint``."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    hint = np.asarray(down_hint, np.float64)
    if abs(float(np.dot(hint, f))) > 0.999:
        hint = np.array([0.0, 0.0, 1.0]) if abs(f[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    x = np.cross(hint, f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ eye
    w2c = np.concatenate([R, t[:, None]], axis=1).astype(np.float32)
    foc = _focal(height, fov_y_deg)
    return Camera(width, height, foc, foc, width / 2.0, height / 2.0, w2c)


def camera_front(width: int, height: int, eye=(0.5, 0.5, -1.5), fov_y_deg: float = 50.0) -> Camera:
    """Axis-aligned camera looking along +z (world axes = camera axes)."""
    eye = np.asarray(eye, np.float64)
    return camera_lookat(width, height, eye, eye + np.array([0.0, 0.0, 1.0]), fov_y_deg)


def camera_on_sphere(rng: np.random.Generator, width: int, height: int, radius: float = 2.0,
                     center=(0.5, 0.5, 0.5), fov_y_deg: float = 50.0) -> Camera:
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    c = np.asarray(center, np.float64)
    return camera_lookat(width, height, c + radius * d, c, fov_y_deg)


# --------------------------------------------------------------------------
# primitive attributes

def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _angles(rng: np.random.Generator, n: int, K: int) -> np.ndarray:
    """Sorted U[0, 2 pi) polar angles, rows resampled until every cyclic gap
    is at most pi - 0.05."""
    th = np.sort(rng.uniform(0.0, TWO_PI, size=(n, K)), axis=1)
    while True:
        gaps = np.diff(np.concatenate([th, th[:, :1] + TWO_PI], axis=1), axis=1)
        bad = np.nonzero(gaps.max(axis=1) > MAX_GAP)[0]
        if bad.size == 0:
            return th
        th[bad] = np.sort(rng.uniform(0.0, TWO_PI, size=(bad.size, K)), axis=1)


def _uniform_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _sh_colors(rng: np.random.Generator, n: int, sh_degree: int) -> np.ndarray:
    if sh_degree < 0:
        return rng.uniform(0.0, 1.0, size=(n, 3))
    ncoef = (sh_degree + 1) ** 2
    c = rng.normal(0.0, 0.05, size=(n, ncoef, 3))
    c[:, 0, :] = rng.uniform(-0.5 / SH_DC_SCALE, 0.5 / SH_DC_SCALE, size=(n, 3))
    return c


def _common(rng, n, K, sh_degree, tau_lo=0.0, tau_hi=1.0):
    scale = np.exp(rng.normal(-3.0, 0.5, size=(n, K)))
    theta = _angles(rng, n, K)
    eta = rng.uniform(0.0, 1.0, size=n)
    tau = -0.1 + 1.09 * rng.uniform(tau_lo, tau_hi, size=n)
    opacity = _sigmoid(rng.standard_normal(n))
    color = _sh_colors(rng, n, sh_degree)
    return scale, theta, eta, tau, opacity, color


def _pack(mu, quat, scale, theta, eta, tau, opacity, color, sh_degree) -> Scene:
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(f(mu), f(quat), f(scale), f(theta), f(eta), f(tau), f(opacity), f(color), sh_degree)


def scene_plain(n: int = 2000, K: int = 8, seed: int = 1000, sh_degree: int = -1) -> Scene:
    """Centres uniform in the unit cube, uniform rotations, plain RGB colour."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0.0, 1.0, size=(n, 3))
    quat = _uniform_quats(rng, n)
    rest = _common(rng, n, K, sh_degree)
    return _pack(mu, quat, *rest, sh_degree)


def _quat_from_matrices(R: np.ndarray) -> np.ndarray:
    from scipy.spatial.transform import Rotation
    xyzw = Rotation.from_matrix(R).as_quat()
    return np.concatenate([xyzw[:, 3:4], xyzw[:, :3]], axis=1)


def _rotvec_matrices(axis_angle: np.ndarray) -> np.ndarray:
    from scipy.spatial.transform import Rotation
    return Rotation.from_rotvec(axis_angle).as_matrix()


def scene_clustered(n: int = 100_000, K: int = 8, seed: int = 2000, n_clusters: int | None = None,
                    bg_frac: float = 0.1, sh_degree: int = 3) -> Scene:
    """Planar surface clusters (90 %) plus a uniform background (10 %).

    Cluster centres ~ U[0.1, 0.9]^3 with uniformly random normals; members lie
    in the cluster plane within +-0.15 of the centre, 0.002 normal jitter,
    random in-plane rotation and a N(0, 0.05 rad) tilt.  Two clusters per
    thousand primitives by default (200 at 100k).
    """
    rng = np.random.default_rng(seed)
    if n_clusters is None:
        n_clusters = max(1, int(round(2 * n / 1000)))
    n_bg = int(round(bg_frac * n))
    n_cl = n - n_bg
    centers = rng.uniform(0.1, 0.9, size=(n_clusters, 3))
    normals = rng.standard_normal((n_clusters, 3))
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    helper = np.where(np.abs(normals[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    t1 = np.cross(normals, helper)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(normals, t1)
    frames = np.stack([t1, t2, normals], axis=2)            # columns t1, t2, n

    cid = rng.integers(0, n_clusters, size=n_cl)
    a = rng.uniform(-0.15, 0.15, size=n_cl)
    b = rng.uniform(-0.15, 0.15, size=n_cl)
    h = rng.normal(0.0, 0.002, size=n_cl)
    mu_cl = centers[cid] + a[:, None] * t1[cid] + b[:, None] * t2[cid] + h[:, None] * normals[cid]
    psi = rng.uniform(0.0, TWO_PI, size=n_cl)
    inplane = _rotvec_matrices(psi[:, None] * np.array([[0.0, 0.0, 1.0]]))
    beta = rng.uniform(0.0, TWO_PI, size=n_cl)
    tilt_axis = np.cos(beta)[:, None] * t1[cid] + np.sin(beta)[:, None] * t2[cid]
    tilt = _rotvec_matrices(rng.normal(0.0, 0.05, size=n_cl)[:, None] * tilt_axis)
    R_cl = tilt @ frames[cid] @ inplane
    quat_cl = _quat_from_matrices(R_cl)

    mu_bg = rng.uniform(0.0, 1.0, size=(n_bg, 3))
    quat_bg = _uniform_quats(rng, n_bg)
    mu = np.concatenate([mu_cl, mu_bg])
    quat = np.concatenate([quat_cl, quat_bg])
    rest = _common(rng, n, K, sh_degree)
    return _pack(mu, quat, *rest, sh_degree)


def scene_slab(n: int = 2_000_000, K: int = 16, seed: int = 5000, sh_degree: int = 3) -> Scene:
    """Heavy depth overlap: x, y ~ U[0, 1], z ~ U[0.25, 0.75]; sharpness drawn
    from the top 5 % of its range (near-hard edges)."""
    rng = np.random.default_rng(seed)
    mu = np.stack([rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(0.25, 0.75, n)], axis=1)
    quat = _uniform_quats(rng, n)
    rest = _common(rng, n, K, sh_degree, tau_lo=0.95, tau_hi=1.0)
    return _pack(mu, quat, *rest, sh_degree)


def scene_layers(n: int = 64, K: int = 8, seed: int = 3100, width: int = 32, height: int = 32,
                 sh_degree: int = 3, max_opacity: float = 0.95):
    """Depth-separated, nearly fronto-facing primitives for derivative checks.

    Returns (scene, camera).  Every primitive has its own centre depth (spaced
    0.8 / n apart) and a tilt of at most 0.008 rad out of the image plane, so
    within the support no two primitives' ray depths cross and the rendered
    image is a smooth function of the parameters almost everywhere.  The
    in-plane rotation is uniform.
    """
    rng = np.random.default_rng(seed)
    cam = camera_front(width, height, eye=(0.5, 0.5, -1.5))
    order = rng.permutation(n)
    z = 0.1 + 0.8 * (order + 0.5) / n
    mu = np.stack([rng.uniform(0.3, 0.7, n), rng.uniform(0.3, 0.7, n), z], axis=1)
    inplane = _rotvec_matrices(rng.uniform(0.0, TWO_PI, n)[:, None] * np.array([[0.0, 0.0, 1.0]]))
    beta = rng.uniform(0.0, TWO_PI, n)
    axis = np.stack([np.cos(beta), np.sin(beta), np.zeros(n)], axis=1)
    tilt = _rotvec_matrices(rng.uniform(0.0, 0.008, n)[:, None] * axis)
    quat = _quat_from_matrices(tilt @ inplane)
    scale = np.exp(rng.normal(-2.7, 0.3, size=(n, K)))
    theta = _angles(rng, n, K)
    eta = rng.uniform(0.05, 0.95, size=n)
    tau = -0.1 + 1.09 * rng.uniform(0.0, 0.8, size=n)
    opacity = np.minimum(_sigmoid(rng.standard_normal(n)), max_opacity)
    color = _sh_colors(rng, n, sh_degree)
    return _pack(mu, quat, scale, theta, eta, tau, opacity, color, sh_degree), cam


# --------------------------------------------------------------------------
# workloads

WORKLOADS = {
    # name: (scene factory, camera factory)
    "plain-2k-128": (lambda: scene_plain(2000, 8, 1000), lambda: camera_front(128, 128)),
    "clustered-100k-1080p": (lambda: scene_clustered(100_000, 8, 2000), lambda: camera_front(1920, 1080)),
    # same scene at a quarter of the pixels (small case for counter captures)
    "clustered-100k-540p": (lambda: scene_clustered(100_000, 8, 2000), lambda: camera_front(960, 540)),
    "train-300k-1600x1064": (lambda: scene_clustered(300_000, 8, 3000), lambda: camera_front(1600, 1064)),
    "slab-2M-k16-4k": (lambda: scene_slab(2_000_000, 16, 5000), lambda: camera_front(3840, 2160)),
}

SERVE_SCENE_SIZES = (50_000, 50_000, 100_000, 100_000, 200_000, 200_000, 500_000, 500_000)
SERVE_RESOLUTIONS = ((640, 480), (1280, 720), (1920, 1080), (3840, 2160))
SERVE_RES_WEIGHTS = (4, 3, 2, 1)


def serve_scenes(sizes=SERVE_SCENE_SIZES, K: int = 8, seed0: int = 4001):
    return [scene_clustered(n, K, seed0 + i) for i, n in enumerate(sizes)]


def serve_requests(count: int, n_scenes: int, rate_hz: float, seed: int = 4500,
                   resolutions=SERVE_RESOLUTIONS, weights=SERVE_RES_WEIGHTS):
    """Poisson arrivals: list of (arrival_s, scene_id, Camera)."""
    rng = np.random.default_rng(seed)
    p = np.asarray(weights, np.float64)
    p /= p.sum()
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate_hz) if rate_hz > 0 else 0.0
        w, h = resolutions[int(rng.choice(len(resolutions), p=p))]
        out.append((t, int(rng.integers(0, n_scenes)), camera_on_sphere(rng, w, h)))
    return out


def raw_scene(n: int, K: int = 8, seed: int = 6000, sh_degree: int = -1, lo=(-0.3, -0.3, 0.4),
              hi=(1.3, 1.3, 0.6)) -> dict:
    """Initial unconstrained (raw) parameters for fitting, drawn in raw
    space: centres uniform in the box [lo, hi], raw quaternions near the
    identity (primitives roughly facing camera_front), raw scales around
    log 0.06, raw angles, blend and sharpness standard normal x 0.3, raw
    opacity around -1, colours uniform (or small SH coefficients)."""
    rng = np.random.default_rng(seed)
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    quat = np.zeros((n, 4))
    quat[:, 0] = 1.0
    quat += rng.normal(0.0, 0.2, size=(n, 4))
    return dict(mu=f(rng.uniform(lo, hi, size=(n, 3))), quat=f(quat),
                scale=f(np.log(0.06) + rng.normal(0.0, 0.3, size=(n, K))),
                theta=f(rng.normal(0.0, 0.3, size=(n, K))), eta=f(rng.normal(0.0, 0.3, size=n)),
                tau=f(rng.normal(0.0, 0.3, size=n)), opacity=f(rng.normal(-1.0, 0.3, size=n)),
                color=f(_sh_colors(rng, n, sh_degree)))


def shape_target(height: int, width: int, seed: int = 6100, n_shapes: int = 6) -> np.ndarray:
    """(3, H, W) float32 image of a few filled convex polygons (3 to 7
    vertices, random rotation and anisotropic size, random colour) painted
    over a grey background, later shapes on top."""
    rng = np.random.default_rng(seed)
    img = np.full((3, height, width), 0.35, np.float64)
    ys, xs = np.mgrid[0:height, 0:width]
    px, py = (xs + 0.5) / width, (ys + 0.5) / height
    for _ in range(n_shapes):
        m = int(rng.integers(3, 8))
        ang = rng.uniform(0, 2 * np.pi) + 2 * np.pi * np.arange(m) / m
        sx, sy = rng.uniform(0.08, 0.3, size=2)
        cx, cy = rng.uniform(0.2, 0.8, size=2)
        vx, vy = cx + sx * np.cos(ang), cy + sy * np.sin(ang)
        inside = np.ones((height, width), bool)
        for k in range(m):
            ex, ey = vx[(k + 1) % m] - vx[k], vy[(k + 1) % m] - vy[k]
            inside &= ex * (py - vy[k]) - ey * (px - vx[k]) >= 0.0
        img[:, inside] = rng.uniform(0.0, 1.0, size=(3, 1))
    return img.astype(np.float32)


def mesh_heightfield(nx: int, ny: int, seed: int = 7000, lo=(-0.3, -0.1), hi=(1.3, 1.1), z0: float = 0.6,
                     amp: float = 0.08, triangles: bool = False):
    """A height-field wall facing camera_front: an (nx+1) x (ny+1) vertex
    grid over [lo, hi] in x, y at depth z0 plus a smooth random relief (a sum
    of a few random sinusoids of amplitude amp).  Returns (verts (V, 3)
    float32, faces (F, 4) or (F, 3) int32, counter-clockwise seen from the
    camera side, -z)."""
    rng = np.random.default_rng(seed)
    xs = np.linspace(lo[0], hi[0], nx + 1)
    ys = np.linspace(lo[1], hi[1], ny + 1)
    X, Y = np.meshgrid(xs, ys)
    Z = np.full_like(X, z0)
    for _ in range(5):
        kx, ky = rng.uniform(1.0, 8.0, size=2)
        ph = rng.uniform(0, 2 * np.pi)
        Z += amp / 5 * np.sin(kx * X + ky * Y + ph)
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    i = np.arange(ny)[:, None] * (nx + 1) + np.arange(nx)[None, :]
    a, b, c, d = i.ravel(), i.ravel() + 1, i.ravel() + nx + 2, i.ravel() + nx + 1
    # seen from -z with y down the image, (a, d, c, b) runs counter-clockwise
    # about -z, the normal that faces the camera
    if triangles:
        faces = np.concatenate([np.stack([a, d, c], 1), np.stack([a, c, b], 1)])
    else:
        faces = np.stack([a, d, c, b], 1)
    return verts.astype(np.float32), faces.astype(np.int32)


def mesh_polygons(n: int, max_vertices: int = 8, seed: int = 7100):
    """n separate convex polygons (3 .. max_vertices vertices: regular
    polygons with a random radius, in-plane stretch and rotation, randomly
    oriented) with centres uniform in the unit cube.  Returns (verts,
    faces (n, max_vertices) int32 with -1 padding)."""
    rng = np.random.default_rng(seed)
    verts, faces = [], []
    q = _uniform_quats(rng, n)
    for f in range(n):
        m = int(rng.integers(3, max_vertices + 1))
        ang = rng.uniform(0, 2 * np.pi) + 2 * np.pi * np.arange(m) / m
        r = rng.uniform(0.02, 0.08)
        sx, sy = rng.uniform(0.6, 1.4, size=2)
        w, x, y, z = q[f]
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        local = np.stack([r * sx * np.cos(ang), r * sy * np.sin(ang), np.zeros(m)], axis=1)
        c = rng.uniform(0.0, 1.0, size=3)
        base = len(verts)
        verts.extend(list(c + local @ R.T))
        faces.append(list(range(base, base + m)) + [-1] * (max_vertices - m))
    return np.asarray(verts, np.float32), np.asarray(faces, np.int32)


def mesh_colors(n_faces: int, seed: int = 7200) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.1, 1.0, size=(n_faces, 3)).astype(np.float32)


def target_image(height: int, width: int, seed: int = 3001) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(3, height, width)).astype(np.float32)


def pixel_sample(width: int, height: int, count: int, seed: int, tiles=()) -> np.ndarray:
    """Seeded random pixel coordinates (x, y) plus every pixel of the listed
    16x16 tiles (given as (tile_x, tile_y)); returns int32 (m, 2), unique."""
    rng = np.random.default_rng(seed)
    count = min(count, width * height)
    lin = rng.choice(width * height, size=count, replace=False)
    pts = [np.stack([lin % width, lin // width], axis=1)]
    for tx, ty in tiles:
        xs = np.arange(tx * 16, min(tx * 16 + 16, width))
        ys = np.arange(ty * 16, min(ty * 16 + 16, height))
        gx, gy = np.meshgrid(xs, ys)
        pts.append(np.stack([gx.ravel(), gy.ravel()], axis=1))
    allp = np.unique(np.concatenate(pts).astype(np.int64), axis=0)
    return np.ascontiguousarray(allp.astype(np.int32))
