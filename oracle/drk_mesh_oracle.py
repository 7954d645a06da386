"""FP64 oracle of the conversion of polygon meshes to DRKs (Sec. 5.4
"Converting Mesh to DRK" and the supplementary section of the same name).

TEST INFRASTRUCTURE ONLY.  Imported by the test-suite; never by the product
path.  Plain numpy; it shares no code with the CUDA library.

Readings (the paper describes the conversion in one sentence: endpoints at
the polygon vertices, tau and eta set for sharpness, "L1 and L2 curvature
set to 1", no optimisation):
  M1  one DRK per face; faces are rows of vertex indices, -1 padding at the
      end of a row.  mu = mean of the face's vertices; plane normal R_z by
      Newell's method (sum over the edges of (v_j - mu) x (v_{j+1} - mu),
      normalised), so the vertices run counter-clockwise about R_z; R_x
      points from mu to the first vertex projected into the plane; R_y =
      R_z x R_x; q is the unit quaternion (w, x, y, z) of [R_x R_y R_z]
      (sign: w >= 0).
  M2  basis endpoints are the vertices projected into the plane, in face
      order.  A face with m < K vertices gets K - m extra endpoints on its
      edges: edge j (from vertex j to j+1) receives floor((K-m)/m) + [j <
      (K-m) mod m] of them at equal spacing.  Collinear endpoints keep the
      L1 contour (Eq. 7) on the same straight edge.
  M3  "L1 and L2 curvature set to 1" is read as eta = 1 (the L1 term of
      Eq. 8 alone), which makes every contour of g a scaled copy of the
      polygon.  The endpoints are scaled by 1/sqrt(-2 ln g_e) so that the
      polygon itself is the contour g = g_e.  g_e = 1/2 (default) puts the
      edges where Psi(g) = 1/2 for every tau (Eq. 9 maps 1/2 to 1/2);
      g_e = exp(-1/2) puts the endpoints exactly on the vertices.
  M4  theta_0 = 0 and theta_k = atan2(endpoint_k . R_y, endpoint_k . R_x) in
      [0, 2 pi); s_k = |endpoint_k| / sqrt(-2 ln g_e).
  M5  tau and opacity as given; colour = base colour x (ambient + diffuse
      |R_z . l|) with a unit light direction l (the supplement shades each
      kernel's base colour with its normal under a predefined light);
      plain RGB.
  M6  a face is rejected with status 1 (an index out of range, fewer than 3
      vertices, or a normal or first-endpoint length below 1e-12 of the
      face size) or status 2 (its endpoint angles do not increase strictly
      with every cyclic gap below pi - 1e-3: not convex enough about mu);
      its DRK gets opacity 0, mu at the origin, the identity rotation,
      equally spaced angles and lengths 1e-3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAP_MARGIN = 1e-3


@dataclass
class MeshOptions:
    K: int = 4
    edge_density: float = 0.5
    tau: float = 0.95
    opacity: float = 1.0
    light: tuple = (0.3, -0.5, -0.8)
    ambient: float = 0.35
    diffuse: float = 0.65


def quat_from_matrix(R: np.ndarray) -> np.ndarray:
    """Unit quaternion (w, x, y, z), w >= 0, of a rotation matrix whose
    columns are the rotated axes (Shepperd's choice of the largest of
    w, x, y, z to divide by)."""
    t = np.trace(R)
    cand = [t, R[0, 0], R[1, 1], R[2, 2]]
    i = int(np.argmax(cand))
    if i == 0:
        w = 0.5 * math.sqrt(1.0 + t)
        q = np.array([w, (R[2, 1] - R[1, 2]) / (4 * w), (R[0, 2] - R[2, 0]) / (4 * w), (R[1, 0] - R[0, 1]) / (4 * w)])
    elif i == 1:
        x = 0.5 * math.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2])
        q = np.array([(R[2, 1] - R[1, 2]) / (4 * x), x, (R[0, 1] + R[1, 0]) / (4 * x), (R[0, 2] + R[2, 0]) / (4 * x)])
    elif i == 2:
        y = 0.5 * math.sqrt(1.0 - R[0, 0] + R[1, 1] - R[2, 2])
        q = np.array([(R[0, 2] - R[2, 0]) / (4 * y), (R[0, 1] + R[1, 0]) / (4 * y), y, (R[1, 2] + R[2, 1]) / (4 * y)])
    else:
        z = 0.5 * math.sqrt(1.0 - R[0, 0] - R[1, 1] + R[2, 2])
        q = np.array([(R[1, 0] - R[0, 1]) / (4 * z), (R[0, 2] + R[2, 0]) / (4 * z), (R[1, 2] + R[2, 1]) / (4 * z), z])
    q /= np.linalg.norm(q)
    return -q if q[0] < 0 else q


def face_endpoints(m: int, K: int, pts: np.ndarray) -> np.ndarray:
    """K endpoints from the m face points (M2)."""
    extra = K - m
    out = []
    for j in range(m):
        a, b = pts[j], pts[(j + 1) % m]
        c = extra // m + (1 if j < extra % m else 0)
        out.append(a)
        for i in range(1, c + 1):
            out.append(a + (b - a) * (i / (c + 1)))
    return np.array(out)


def convert_face(V: np.ndarray, face: np.ndarray, base: np.ndarray, opt: MeshOptions):
    """(params dict of one DRK, status) for one face."""
    K = opt.K
    row = [int(i) for i in face]
    m = 0
    while m < len(row) and row[m] >= 0:
        m += 1
    idx = row[:m]
    reject = {"mu": np.zeros(3), "quat": np.array([1.0, 0, 0, 0]), "scale": np.full(K, 1e-3),
              "theta": 2 * math.pi * np.arange(K) / K, "eta": 1.0, "tau": opt.tau, "opacity": 0.0,
              "color": np.zeros(3)}
    if m < 3 or m > K or any(i >= len(V) for i in idx) or any(r >= 0 for r in row[m:]):
        return reject, 1
    P = V[idx]
    mu = P.mean(axis=0)
    size = max(np.linalg.norm(P - mu, axis=1).max(), 1e-300)
    n = np.zeros(3)
    for j in range(m):
        n += np.cross(P[j] - mu, P[(j + 1) % m] - mu)
    nn = np.linalg.norm(n)
    if nn <= 1e-12 * size * size:
        return reject, 1
    Rz = n / nn
    d0 = P[0] - mu
    d0 = d0 - Rz * (d0 @ Rz)
    l0 = np.linalg.norm(d0)
    if l0 <= 1e-12 * size:
        return reject, 1
    Rx = d0 / l0
    Ry = np.cross(Rz, Rx)
    loc = np.stack([(P - mu) @ Rx, (P - mu) @ Ry], axis=1)       # projected into the plane
    E = face_endpoints(m, K, loc)
    th = np.zeros(K)
    for k in range(1, K):
        a = math.atan2(E[k, 1], E[k, 0])
        th[k] = a + 2 * math.pi if a < 0 else a
    gaps = np.diff(np.append(th, 2 * math.pi))
    if np.any(gaps <= 0) or np.any(gaps >= math.pi - GAP_MARGIN):
        return reject, 2
    f = 1.0 / math.sqrt(-2.0 * math.log(opt.edge_density))
    R = np.stack([Rx, Ry, Rz], axis=1)
    l = np.asarray(opt.light, np.float64)
    l = l / np.linalg.norm(l)
    shade = opt.ambient + opt.diffuse * abs(Rz @ l)
    return {"mu": mu, "quat": quat_from_matrix(R), "scale": np.linalg.norm(E, axis=1) * f, "theta": th,
            "eta": 1.0, "tau": opt.tau, "opacity": opt.opacity, "color": np.asarray(base, np.float64) * shade}, 0


def mesh_to_drk(verts, faces, face_color, opt: MeshOptions):
    """Arrays of the converted DRKs (float64, shapes of a scene with
    sh_degree -1) and the per-face status."""
    V = np.asarray(verts, np.float64)
    F = np.asarray(faces, np.int64)
    Cb = np.asarray(face_color, np.float64)
    out = {k: [] for k in ("mu", "quat", "scale", "theta", "eta", "tau", "opacity", "color")}
    status = np.zeros(len(F), np.int32)
    for f in range(len(F)):
        p, st = convert_face(V, F[f], Cb[f], opt)
        status[f] = st
        for k in out:
            out[k].append(p[k])
    return {k: np.array(v, np.float64) for k, v in out.items()}, status
