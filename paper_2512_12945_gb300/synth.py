"""Seeded synthetic inputs shaped like the paper's workloads.

The paper evaluates on SemanticKITTI (64-beam LiDAR, 10 cm voxels) and
SceneNet RGB-D (640x480 depth, 5 cm / 10 cm voxels) with network-predicted
semantics (Sec. IV). Neither dataset nor any network is available, so these
generators stand in for them: analytic ray casting of seeded primitive scenes
(planes, boxes, spheres, vertical cylinders), a spinning-LiDAR or pinhole
depth sensor, a seeded trajectory, and per-point class probabilities or
embeddings drawn around the true object class.

This module holds none of the method's arithmetic (no transform, no band
traversal, no fusion). It serves the CUDA path, the oracle and the benchmark
alike; every array it returns is plain numpy (float32 points and semantics,
float64 poses).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------- scene
@dataclass
class Scene:
    planes: list = field(default_factory=list)     # (normal(3), offset, obj)
    boxes: list = field(default_factory=list)      # (lo(3), hi(3), obj)
    spheres: list = field(default_factory=list)    # (centre(3), radius, obj)
    cylinders: list = field(default_factory=list)  # (cx, cy, radius, z0, z1, obj)

    def n_objects(self):
        ids = [p[-1] for p in self.planes + self.boxes + self.spheres + self.cylinders]
        return max(ids) + 1 if ids else 0

    def raycast(self, origin, dirs):
        """Nearest hit distance t (inf on a miss) and object id (-1) per ray."""
        o = np.asarray(origin, np.float64).reshape(1, 3)
        d = np.asarray(dirs, np.float64)
        n = d.shape[0]
        best = np.full(n, np.inf)
        obj = np.full(n, -1, np.int64)
        eps = 1e-6

        def take(t, oid):
            m = (t > eps) & (t < best)
            best[m] = t[m]
            obj[m] = oid

        with np.errstate(divide="ignore", invalid="ignore"):
            for nrm, off, oid in self.planes:
                nrm = np.asarray(nrm, np.float64)
                den = d @ nrm
                t = (off - float(o[0] @ nrm)) / den
                t[~np.isfinite(t)] = np.inf
                take(t, oid)
            for lo, hi, oid in self.boxes:
                lo = np.asarray(lo, np.float64)
                hi = np.asarray(hi, np.float64)
                inv = 1.0 / d
                t1 = (lo - o) * inv
                t2 = (hi - o) * inv
                tmin = np.nanmax(np.minimum(t1, t2), axis=1)
                tmax = np.nanmin(np.maximum(t1, t2), axis=1)
                hit = tmax >= np.maximum(tmin, 0.0)
                t = np.where(tmin > eps, tmin, tmax)
                t = np.where(hit, t, np.inf)
                take(t, oid)
            for c, rad, oid in self.spheres:
                oc = o - np.asarray(c, np.float64)
                b = d @ oc[0]
                cc = float(oc[0] @ oc[0]) - rad * rad
                disc = b * b - cc
                sq = np.sqrt(np.maximum(disc, 0.0))
                t = np.where(-b - sq > eps, -b - sq, -b + sq)
                t = np.where(disc >= 0, t, np.inf)
                take(t, oid)
            for cx, cy, rad, z0, z1, oid in self.cylinders:
                ox, oy = o[0, 0] - cx, o[0, 1] - cy
                a = d[:, 0] ** 2 + d[:, 1] ** 2
                b = ox * d[:, 0] + oy * d[:, 1]
                cc = ox * ox + oy * oy - rad * rad
                disc = b * b - a * cc
                sq = np.sqrt(np.maximum(disc, 0.0))
                t = (-b - sq) / a
                t = np.where(t > eps, t, (-b + sq) / a)
                z = o[0, 2] + t * d[:, 2]
                ok = (disc >= 0) & (a > 0) & (z >= z0) & (z <= z1)
                take(np.where(ok, t, np.inf), oid)
        return best, obj


# ------------------------------------------------------------------------- sensors
def lidar_dirs(n_beams, n_az, fov_up_deg, fov_down_deg):
    """Unit ray directions (n_az * n_beams, 3) in the sensor frame, ordered
    azimuth-major: all beams of one azimuth column are contiguous."""
    el = np.deg2rad(np.linspace(fov_up_deg, fov_down_deg, n_beams))
    az = np.arange(n_az) * (2.0 * math.pi / n_az)
    A, E = np.meshgrid(az, el, indexing="ij")
    d = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], axis=-1)
    return d.reshape(-1, 3)


def pinhole_dirs(width, height, focal):
    """Per-pixel rays of a centred pinhole camera (x right, y down, z forward),
    row-major. Returns (unit directions (H*W, 3), z component of each)."""
    u = (np.arange(width) + 0.5 - width / 2.0) / focal
    v = (np.arange(height) + 0.5 - height / 2.0) / focal
    V, U = np.meshgrid(v, u, indexing="ij")
    d = np.stack([U, V, np.ones_like(U)], axis=-1).reshape(-1, 3)
    n = np.linalg.norm(d, axis=1, keepdims=True)
    return d / n, (1.0 / n[:, 0])


def translation(x, y, z):
    m = np.eye(4)
    m[:3, 3] = (x, y, z)
    return m


def rot_z(yaw):
    c, s = math.cos(yaw), math.sin(yaw)
    m = np.eye(4)
    m[:2, :2] = [[c, -s], [s, c]]
    return m


def look_at(eye, target, up=(0.0, 0.0, 1.0)):
    """world_from_camera for a camera at eye looking at target (z forward,
    x right, y down)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    dn = np.cross(f, r)
    m = np.eye(4)
    m[:3, 0] = r
    m[:3, 1] = dn
    m[:3, 2] = f
    m[:3, 3] = eye
    return m


# ------------------------------------------------------------------------ scenes
def room_scene(rng, size=(10.0, 10.0, 3.0), n_objects=6):
    """Room of six planes plus seeded boxes / spheres (objects 6..)."""
    X, Y, Z = size
    sc = Scene()
    sc.planes = [((0, 0, 1), 0.0, 0), ((0, 0, 1), Z, 1), ((1, 0, 0), 0.0, 2),
                 ((1, 0, 0), X, 3), ((0, 1, 0), 0.0, 4), ((0, 1, 0), Y, 5)]
    for k in range(n_objects):
        oid = 6 + k
        c = rng.uniform([1.5, 1.5, 0.3], [X - 1.5, Y - 1.5, 1.5])
        if rng.random() < 0.5:
            h = rng.uniform(0.2, 0.6, size=3)
            lo = c - h
            lo[2] = 0.0
            sc.boxes.append((lo, c + h, oid))
        else:
            sc.spheres.append((c, float(rng.uniform(0.25, 0.6)), oid))
    return sc


def street_scene(rng, length=160.0):
    """Street along +x: ground, box buildings on both sides, poles, cars."""
    sc = Scene()
    sc.planes = [((0, 0, 1), 0.0, 0)]
    oid = 1
    for side in (-1, 1):
        x = -40.0
        while x < length:
            w = rng.uniform(8.0, 25.0)
            setback = rng.uniform(8.0, 14.0)
            depth = rng.uniform(8.0, 15.0)
            h = rng.uniform(6.0, 25.0)
            y0, y1 = (setback, setback + depth) if side > 0 else (-setback - depth, -setback)
            sc.boxes.append(((x, y0, 0.0), (x + w, y1, h), oid))
            oid += 1
            x += w + rng.uniform(1.0, 6.0)
    for side in (-1, 1):
        x = -30.0
        while x < length:
            sc.cylinders.append((x, side * 6.5, 0.15, 0.0, float(rng.uniform(4.0, 8.0)), oid))
            oid += 1
            x += rng.uniform(12.0, 20.0)
    for _ in range(int(length / 6)):
        cx = rng.uniform(-30.0, length)
        cy = rng.choice([-3.5, 3.5]) + rng.uniform(-0.3, 0.3)
        sc.boxes.append(((cx - 2.25, cy - 0.9, 0.0), (cx + 2.25, cy + 0.9, 1.5), oid))
        oid += 1
    return sc


def indoor_scene(rng, size=(6.0, 5.0, 3.0), n_objects=30):
    """Indoor room with seeded furniture-like boxes and spheres."""
    X, Y, Z = size
    sc = Scene()
    sc.planes = [((0, 0, 1), 0.0, 0), ((0, 0, 1), Z, 1), ((1, 0, 0), 0.0, 2),
                 ((1, 0, 0), X, 3), ((0, 1, 0), 0.0, 4), ((0, 1, 0), Y, 5)]
    for k in range(n_objects - 6):
        oid = 6 + k
        c = rng.uniform([0.4, 0.4, 0.1], [X - 0.4, Y - 0.4, 1.8])
        if rng.random() < 0.7:
            h = rng.uniform(0.1, 0.4, size=3)
            lo = c - h
            if rng.random() < 0.6:
                lo[2] = 0.0
            sc.boxes.append((lo, c + h, oid))
        else:
            sc.spheres.append((c, float(rng.uniform(0.1, 0.3)), oid))
    return sc


# --------------------------------------------------------------------- semantics
def dirichlet_probs(rng, labels, K, p_true=0.8, kappa=20.0):
    """Class probabilities ~ Dirichlet(kappa * mu), mu = p_true on the label and
    (1 - p_true)/(K - 1) elsewhere."""
    n = labels.shape[0]
    alpha = np.full((n, K), kappa * (1.0 - p_true) / (K - 1))
    alpha[np.arange(n), labels] = kappa * p_true
    g = rng.standard_gamma(alpha)
    g /= g.sum(axis=1, keepdims=True)
    return g.astype(np.float32)


def flipped_probs(rng, labels, K, p_true=0.7, flip=0.1):
    """p_true on the (possibly flipped) label, the rest spread evenly; a
    fraction `flip` of the points gets a random wrong label."""
    n = labels.shape[0]
    lab = labels.copy()
    f = rng.random(n) < flip
    wrong = (lab[f] + rng.integers(1, K, size=int(f.sum()))) % K
    lab[f] = wrong
    p = np.full((n, K), (1.0 - p_true) / (K - 1), np.float32)
    p[np.arange(n), lab] = p_true
    return p


def unit_centroids(rng, n, dim):
    c = rng.standard_normal((n, dim))
    return c / np.linalg.norm(c, axis=1, keepdims=True)


def embeddings(rng, labels, centroids, sigma=0.1):
    """z = normalize(centroid[label] + N(0, sigma^2 I)), float32."""
    z = centroids[labels] + sigma * rng.standard_normal((labels.shape[0], centroids.shape[1]))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    return z.astype(np.float32)


# ----------------------------------------------------------------------- configs
@dataclass
class Workload:
    name: str
    voxel_size: float
    trunc: float
    min_range: float
    max_range: float
    mode: str                # "onehot" | "soft" | "open"
    num_classes: int
    embed_dim: int
    body_from_sensor: np.ndarray
    scans: list              # list of dict(pts, pose, sem, labels)
    image_width: int = 0     # organized frames: pixels per image row (0: unorganized)

    @property
    def n_points(self):
        return int(sum(s["pts"].shape[0] for s in self.scans))


def _lidar_scan(rng, scene, world_from_sensor, dirs_s, noise, max_range):
    R = world_from_sensor[:3, :3]
    o = world_from_sensor[:3, 3]
    t, obj = scene.raycast(o, dirs_s @ R.T)
    hit = np.isfinite(t) & (t <= max_range)
    rr = t + noise * rng.standard_normal(t.shape[0])
    rr[~hit] = 0.0
    pts = (dirs_s * rr[:, None]).astype(np.float32)
    pts[~hit] = 0.0
    obj[~hit] = 0
    return pts, obj, hit


def room_lidar(seed=1, n_scans=10, n_beams=16, n_az=512, K=10, mode="onehot",
               p_true=0.8, kappa=20.0):
    """Room 10x10x3 m + 6 objects, LiDAR on a circle of radius 2 m at 1.5 m."""
    rng = np.random.default_rng(seed)
    sc = room_scene(rng)
    dirs = lidar_dirs(n_beams, n_az, 15.0, -15.0)
    n_obj = sc.n_objects()
    cls_of = np.array([0, 1, 2, 2, 2, 2] + [3 + (k % (K - 3)) for k in range(n_obj - 6)])
    scans = []
    for s in range(n_scans):
        a = 2.0 * math.pi * s / n_scans
        pose = translation(5.0 + 2.0 * math.cos(a), 5.0 + 2.0 * math.sin(a), 1.5) @ rot_z(a + 0.3)
        pts, obj, hit = _lidar_scan(rng, sc, pose, dirs, 0.01, 100.0)
        lab = cls_of[obj]
        sem = dirichlet_probs(rng, lab, K, p_true, kappa)
        scans.append(dict(pts=pts, pose=pose, sem=sem, labels=lab))
    return Workload("room-lidar", 0.1, 0.3, 0.1, 100.0, mode, K, 0, np.eye(4), scans)


def street_lidar(seed=2, n_scans=100, n_beams=64, n_az=2048, K=20, flip=0.1, p_true=0.7):
    """Urban LiDAR: 64 beams (+2 to -24.9 deg) x n_az azimuths, driving 1 m per
    scan along a seeded street; sensor 1.73 m above the body frame."""
    rng = np.random.default_rng(seed)
    sc = street_scene(rng, length=n_scans + 90.0)
    dirs = lidar_dirs(n_beams, n_az, 2.0, -24.9)
    ext = translation(0.0, 0.0, 1.73)
    # class ids: 0 ground, 1 building, 2 pole, 3.. cars (spread over the rest)
    cls_of = np.zeros(sc.n_objects(), np.int64)
    for lo, hi, oid in sc.boxes:
        cls_of[oid] = 1 if hi[2] > 1.6 else 3 + (oid % (K - 3))
    for cyl in sc.cylinders:
        cls_of[cyl[-1]] = 2
    scans = []
    for s in range(n_scans):
        body = translation(float(s), 0.0, 0.0)
        pts, obj, hit = _lidar_scan(rng, sc, body @ ext, dirs, 0.01, 80.0)
        lab = cls_of[obj]
        sem = flipped_probs(rng, lab, K, p_true, flip)
        scans.append(dict(pts=pts, pose=body, sem=sem, labels=lab))
    return Workload("street-lidar", 0.1, 0.3, 1.0, 80.0, "onehot", K, 0, ext, scans)


def indoor_rgbd(seed=3, n_frames=200, width=640, height=480, focal=525.0, dim=512,
                n_objects=30, sigma=0.1, voxel=0.05, frames=None):
    """Indoor RGB-D: depth frames (row-major pixels) from a smooth camera loop,
    one unit embedding per pixel drawn around its object's centroid.
    `frames` selects a subset of frame indices (same trajectory)."""
    rng = np.random.default_rng(seed)
    sc = indoor_scene(rng, n_objects=n_objects)
    cents = unit_centroids(rng, sc.n_objects(), dim)
    dirs, zc = pinhole_dirs(width, height, focal * width / 640.0)
    scans = []
    sel = range(n_frames) if frames is None else frames
    for f in sel:
        frng = np.random.default_rng([seed, f])
        a = 2.0 * math.pi * f / max(n_frames, 1)
        eye = (3.0 + 1.5 * math.cos(a), 2.5 + 1.2 * math.sin(a), 1.4 + 0.2 * math.sin(2 * a))
        tgt = (3.0 - 1.0 * math.cos(a + 0.8), 2.5 - 1.0 * math.sin(a + 0.8), 0.9)
        pose = look_at(eye, tgt)
        R = pose[:3, :3]
        t, obj = sc.raycast(pose[:3, 3], dirs @ R.T)
        depth = t * zc
        hit = np.isfinite(t) & (depth >= 0.3) & (depth <= 5.0)
        pts = (dirs * np.where(hit, t, 0.0)[:, None]).astype(np.float32)
        obj[~hit] = 0
        sem = embeddings(frng, obj, cents, sigma)
        scans.append(dict(pts=pts, pose=pose, sem=sem, labels=obj))
    return Workload("indoor-rgbd", voxel, 3.0 * voxel, 0.3, 8.0, "open", 0, dim, np.eye(4),
                    scans, image_width=width)


def indoor_centroids(seed=3, dim=512, n_objects=30):
    """The class centroids indoor_rgbd draws for `seed` (after its scene)."""
    rng = np.random.default_rng(seed)
    sc = indoor_scene(rng, n_objects=n_objects)
    return unit_centroids(rng, sc.n_objects(), dim)


def indoor_embeddings_device(labels, centroids, seed, frame, sigma=0.1):
    """Device-side draw of the indoor embeddings for long runs:
    z = normalize(centroid[label] + N(0, sigma^2 I)) per pixel, float32, on
    the device of `labels` (a torch int64 tensor) from a torch generator
    seeded by (seed, frame). Same distribution as `embeddings`, not the same
    numbers."""
    import torch
    dev = labels.device
    g = torch.Generator(device=dev).manual_seed(int(seed) * 100003 + int(frame))
    c = torch.as_tensor(centroids, dtype=torch.float32, device=dev)
    z = c[labels] + sigma * torch.randn((labels.shape[0], c.shape[1]), device=dev, generator=g)
    z /= torch.linalg.vector_norm(z, dim=1, keepdim=True)
    return z.contiguous()


def random_queries(seed, n, dim):
    """n seeded random unit query vectors (float32)."""
    rng = np.random.default_rng(seed)
    return unit_centroids(rng, n, dim).astype(np.float32)


def batch_workload(seed=5, n_scans=10):
    """The batched multi-map configuration: 8 closed-set street maps (64 beams,
    azimuth counts drawn from [320, 3900), so 20 k-250 k points per scan) and
    8 open-set RGB-D maps (l = 256, 320 x 240 to 640 x 480), n_scans scans
    each. Returns (closed workloads, open workloads)."""
    rng = np.random.default_rng(seed)
    closed = []
    for k in range(8):
        n_az = int(rng.integers(320, 3900))
        closed.append(street_lidar(seed=50 + k, n_scans=n_scans, n_az=n_az))
    sizes = [(320, 240), (400, 300), (480, 360), (640, 480)] * 2
    opened = [indoor_rgbd(seed=60 + k, n_frames=40, width=wd, height=ht, dim=256,
                          frames=list(range(n_scans))) for k, (wd, ht) in enumerate(sizes)]
    return closed, opened
