"""Seeded synthetic scenes shaped like the workloads of KISS-Matcher (arXiv
2409.15615): scan-level LiDAR pairs (Sec. IV-A, 64-channel scans of 10K-30K
voxelised points, Sec. III-C) and dense, map-sized clouds (Sec. IV-B).

The paper's datasets (KITTI, MulRan, Kimera-Multi) are not available, so every
cloud here is drawn from a seeded generator:

* ``scene_pair``  - 10 m cube with three axis-aligned planes, four spheres and
  three vertical cylinders, sampled uniformly by area with Gaussian noise; the
  target is an independent resample cropped to the x >= 4 m slab (60 % of the
  source extent) and moved by a uniform random rotation and a translation of
  at most 2 m.
* ``lidar_pair``  - a 64-beam spinning scanner (elevation -25..+3 deg, 2048
  azimuth bins by default, about 120k returns, range <= 80 m, Gaussian range noise) ray-cast into
  a ground plane, 30 boxes, 50 vertical poles and 10 walls; the second scan is
  taken 10 m further along x with a yaw of up to 30 deg.
* ``indoor_pair`` - a 4 x 3 x 2.2 m room (floor and four walls) with 40 box/cylinder
  furniture composites, densely sampled (2M points by default) with 5 mm
  noise; the second cloud is an independent resample under a random rigid
  motion.

Every function returns float32 arrays of shape [n, 3] and the ground-truth
motion (R, t) with target = R @ source + t (Eq. 1 of the paper, noise free).
Only numpy's PCG64 generator is used, so a seed fixes the cloud.
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------------------
# rigid motions
# ----------------------------------------------------------------------------


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (Shoemake's subgroup algorithm, Graphics Gems
    III, 1992): a unit quaternion from three uniform variates."""
    u1, u2, u3 = rng.random(3)
    a = math.sqrt(1.0 - u1)
    b = math.sqrt(u1)
    qx = a * math.sin(2 * math.pi * u2)
    qy = a * math.cos(2 * math.pi * u2)
    qz = b * math.sin(2 * math.pi * u3)
    qw = b * math.cos(2 * math.pi * u3)
    return np.array(
        [
            [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
            [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
            [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)],
        ]
    )


def random_translation(rng: np.random.Generator, max_norm: float) -> np.ndarray:
    """Uniform random point in the ball of radius ``max_norm``."""
    while True:
        t = rng.uniform(-max_norm, max_norm, 3)
        if np.dot(t, t) <= max_norm * max_norm:
            return t


def yaw_matrix(yaw: float) -> np.ndarray:
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _apply(R: np.ndarray, t: np.ndarray, x: np.ndarray) -> np.ndarray:
    return (x @ R.T + t).astype(np.float32)


# ----------------------------------------------------------------------------
# surface primitives sampled uniformly by area
# ----------------------------------------------------------------------------


class _Rect:
    """Axis-aligned rectangle: origin o, edge vectors e1, e2 (orthogonal)."""

    def __init__(self, o, e1, e2):
        self.o = np.asarray(o, float)
        self.e1 = np.asarray(e1, float)
        self.e2 = np.asarray(e2, float)

    def area(self):
        return float(np.linalg.norm(self.e1) * np.linalg.norm(self.e2))

    def sample(self, rng, n):
        s = rng.random((n, 2))
        return self.o + s[:, :1] * self.e1 + s[:, 1:] * self.e2


class _Sphere:
    def __init__(self, c, r):
        self.c = np.asarray(c, float)
        self.r = float(r)

    def area(self):
        return 4 * math.pi * self.r ** 2

    def sample(self, rng, n):
        d = rng.standard_normal((n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        return self.c + self.r * d


class _Cylinder:
    """Vertical cylinder (lateral surface plus top cap) standing at base c."""

    def __init__(self, c, r, h):
        self.c = np.asarray(c, float)
        self.r = float(r)
        self.h = float(h)

    def area(self):
        return 2 * math.pi * self.r * self.h + math.pi * self.r ** 2

    def sample(self, rng, n):
        lat = 2 * math.pi * self.r * self.h
        on_side = rng.random(n) < lat / self.area()
        phi = rng.uniform(0, 2 * math.pi, n)
        out = np.empty((n, 3))
        z = rng.uniform(0, self.h, n)
        rr = self.r * np.sqrt(rng.random(n))
        rad = np.where(on_side, self.r, rr)
        out[:, 0] = self.c[0] + rad * np.cos(phi)
        out[:, 1] = self.c[1] + rad * np.sin(phi)
        out[:, 2] = self.c[2] + np.where(on_side, z, self.h)
        return out


class _Box:
    """Axis-aligned box surface (all six faces)."""

    def __init__(self, lo, hi):
        lo = np.asarray(lo, float)
        hi = np.asarray(hi, float)
        ex = np.array([hi[0] - lo[0], 0, 0])
        ey = np.array([0, hi[1] - lo[1], 0])
        ez = np.array([0, 0, hi[2] - lo[2]])
        self.faces = [
            _Rect(lo, ex, ey), _Rect(lo + ez, ex, ey),
            _Rect(lo, ex, ez), _Rect(lo + ey, ex, ez),
            _Rect(lo, ey, ez), _Rect(lo + ex, ey, ez),
        ]

    def area(self):
        return sum(f.area() for f in self.faces)

    def sample(self, rng, n):
        return _sample_mixture(self.faces, rng, n)


def _sample_mixture(prims, rng, n):
    areas = np.array([p.area() for p in prims])
    counts = rng.multinomial(n, areas / areas.sum())
    parts = [p.sample(rng, int(c)) for p, c in zip(prims, counts) if c > 0]
    pts = np.concatenate(parts, axis=0)
    return pts[rng.permutation(len(pts))]


def _sample_region(prims, rng, n, keep=None, sigma=0.0):
    """n noisy surface samples, optionally restricted by a predicate."""
    out = []
    have = 0
    while have < n:
        m = max(2 * (n - have), 1024)
        pts = _sample_mixture(prims, rng, m)
        if sigma > 0:
            pts = pts + rng.normal(0.0, sigma, pts.shape)
        if keep is not None:
            pts = pts[keep(pts)]
        out.append(pts)
        have += len(pts)
    return np.concatenate(out, axis=0)[:n]


# ----------------------------------------------------------------------------
# scene pair: planes, spheres, cylinders in a 10 m cube
# ----------------------------------------------------------------------------


def _cube_scene(rng):
    L = 10.0
    prims = [
        _Rect([0, 0, 0], [L, 0, 0], [0, L, 0]),  # floor z = 0
        _Rect([0, 0, 0], [0, L, 0], [0, 0, L]),  # wall x = 0
        _Rect([0, 0, 0], [L, 0, 0], [0, 0, L]),  # wall y = 0
    ]
    for _ in range(4):
        r = rng.uniform(0.3, 1.0)
        c = [rng.uniform(1.5, 8.5), rng.uniform(1.5, 8.5), rng.uniform(r + 0.5, 6.0)]
        prims.append(_Sphere(c, r))
    for _ in range(3):
        r = rng.uniform(0.2, 0.5)
        h = rng.uniform(1.0, 4.0)
        prims.append(_Cylinder([rng.uniform(1.0, 9.0), rng.uniform(1.0, 9.0), 0.0], r, h))
    return prims


def _clutter_scene(rng, n_spheres=12, n_boxes=8):
    """Cube-scene objects without the three large planes, plus extra spheres
    and boxes: a scene whose points are mostly distinctive (the role the
    paper's geometric suppression plays for plane-dominated scans)."""
    prims = _cube_scene(rng)[3:]
    for _ in range(n_spheres):
        r = rng.uniform(0.3, 1.0)
        prims.append(_Sphere([rng.uniform(1, 9), rng.uniform(1, 9), rng.uniform(0.5, 6)], r))
    for _ in range(n_boxes):
        lo = rng.uniform(0, 8, 3)
        prims.append(_Box(lo, lo + rng.uniform(0.3, 1.5, 3)))
    return prims


def scene_pair(seed: int, n: int = 20000, sigma: float = 0.01, crop_x: float = 4.0,
               max_t: float = 2.0, clutter: bool = False):
    """Source/target pair from the 10 m cube scene (``clutter=True``: the
    plane-free, object-rich variant).

    Returns ``(src, tgt, R, t, vp_src, vp_tgt)``; the viewpoints are the cube
    centre expressed in each cloud's frame (used to orient normals).
    """
    rng = np.random.default_rng(seed)
    prims = _clutter_scene(rng) if clutter else _cube_scene(rng)
    src = _sample_region(prims, rng, n, sigma=sigma)
    tgt_w = _sample_region(prims, rng, n, keep=lambda p: p[:, 0] >= crop_x, sigma=sigma)
    R = random_rotation(rng)
    t = random_translation(rng, max_t)
    tgt = _apply(R, t, tgt_w)
    vp = np.array([5.0, 5.0, 5.0])
    return src.astype(np.float32), tgt, R, t, vp, R @ vp + t


# ----------------------------------------------------------------------------
# LiDAR pair: ray casting a 64-beam scanner into a street-like scene
# ----------------------------------------------------------------------------


class _LidarScene:
    def __init__(self, rng, extent=70.0, clear=4.0):
        boxes = []  # (cx, cy, yaw, hx, hy, h)
        def ok(cx, cy, rad):
            # keep the sensor path y ~ 0, x in [-5, 15] free
            return not (-8 - rad < cx < 18 + rad and abs(cy) < clear + rad)
        while len(boxes) < 30:
            cx, cy = rng.uniform(-extent, extent, 2)
            hx, hy = rng.uniform(0.5, 2.5, 2)
            if ok(cx, cy, max(hx, hy) * 1.5):
                boxes.append((cx, cy, rng.uniform(0, math.pi), hx, hy, rng.uniform(1.0, 4.0)))
        walls = []
        while len(walls) < 10:
            cx, cy = rng.uniform(-extent, extent, 2)
            hx = rng.uniform(5.0, 20.0)
            if ok(cx, cy, hx):
                walls.append((cx, cy, rng.uniform(0, math.pi), hx, 0.15, rng.uniform(3.0, 6.0)))
        poles = []
        while len(poles) < 50:
            cx, cy = rng.uniform(-extent, extent, 2)
            if ok(cx, cy, 0.5):
                poles.append((cx, cy, rng.uniform(0.1, 0.3), rng.uniform(3.0, 8.0)))
        self.boxes = np.array(boxes + walls)
        self.poles = np.array(poles)

    def cast(self, o, d, max_range):
        """Nearest hit distance along unit rays d (n,3) from origin o (3,)."""
        n = d.shape[0]
        best = np.full(n, np.inf)
        # ground plane z = 0
        with np.errstate(divide="ignore", invalid="ignore"):
            tg = np.where(d[:, 2] < -1e-9, -o[2] / d[:, 2], np.inf)
        best = np.minimum(best, tg)
        # oriented boxes (yaw about z), bottom at z = 0
        for cx, cy, yaw, hx, hy, h in self.boxes:
            c, s = math.cos(yaw), math.sin(yaw)
            ox, oy = o[0] - cx, o[1] - cy
            lo_x = c * ox + s * oy
            lo_y = -s * ox + c * oy
            ld_x = c * d[:, 0] + s * d[:, 1]
            ld_y = -s * d[:, 0] + c * d[:, 1]
            tmin = np.zeros(n)
            tmax = np.full(n, np.inf)
            for lo, ld, hw_lo, hw_hi in ((lo_x, ld_x, -hx, hx), (lo_y, ld_y, -hy, hy),
                                         (o[2], d[:, 2], 0.0, h)):
                with np.errstate(divide="ignore", invalid="ignore"):
                    inv = 1.0 / ld
                    t1 = (hw_lo - lo) * inv
                    t2 = (hw_hi - lo) * inv
                tn = np.minimum(t1, t2)
                tf = np.maximum(t1, t2)
                par = np.abs(ld) < 1e-12
                inside = (lo >= hw_lo) & (lo <= hw_hi)
                tn = np.where(par, np.where(inside, -np.inf, np.inf), tn)
                tf = np.where(par, np.where(inside, np.inf, -np.inf), tf)
                tmin = np.maximum(tmin, tn)
                tmax = np.minimum(tmax, tf)
            hit = (tmax >= tmin) & (tmin > 1e-6)
            best = np.where(hit, np.minimum(best, tmin), best)
        # vertical poles
        for cx, cy, r, h in self.poles:
            ox, oy = o[0] - cx, o[1] - cy
            a = d[:, 0] ** 2 + d[:, 1] ** 2
            b = 2 * (ox * d[:, 0] + oy * d[:, 1])
            cc = ox * ox + oy * oy - r * r
            disc = b * b - 4 * a * cc
            with np.errstate(invalid="ignore", divide="ignore"):
                tc = (-b - np.sqrt(disc)) / (2 * a)
            z = o[2] + tc * d[:, 2]
            hit = (disc >= 0) & (a > 1e-12) & (tc > 1e-6) & (z >= 0) & (z <= h)
            best = np.where(hit, np.minimum(best, tc), best)
        best[best > max_range] = np.inf
        return best


def _scan(scene, rng, pos, yaw, beams, az_bins, max_range, sigma, height):
    elev = np.deg2rad(np.linspace(-25.0, 3.0, beams))
    az = 2 * math.pi * (np.arange(az_bins) + 0.5) / az_bins
    ee, aa = np.meshgrid(elev, az, indexing="ij")
    d_s = np.stack([np.cos(ee) * np.cos(aa), np.cos(ee) * np.sin(aa), np.sin(ee)], -1).reshape(-1, 3)
    Rw = yaw_matrix(yaw)
    o = np.array([pos[0], pos[1], height])
    d_w = d_s @ Rw.T
    rng_hit = scene.cast(o, d_w, max_range)
    ok = np.isfinite(rng_hit)
    r = rng_hit[ok] + rng.normal(0.0, sigma, int(ok.sum()))
    pts_s = d_s[ok] * r[:, None]  # sensor frame
    return pts_s, Rw, o


def lidar_pair(seed: int, beams: int = 64, az_bins: int = 2048, max_range: float = 80.0,
               sigma: float = 0.02, travel: float = 10.0, max_yaw_deg: float = 30.0,
               height: float = 1.73):
    """Two scans of one street-like scene.

    Returns ``(src, tgt, R, t, vp_src, vp_tgt)``; points are in each sensor's
    frame and the viewpoints are the sensor origins.
    """
    rng = np.random.default_rng(seed)
    scene = _LidarScene(rng)
    yaw2 = math.radians(rng.uniform(-max_yaw_deg, max_yaw_deg))
    p1, R1, o1 = _scan(scene, rng, (0.0, 0.0), 0.0, beams, az_bins, max_range, sigma, height)
    p2, R2, o2 = _scan(scene, rng, (travel, 0.0), yaw2, beams, az_bins, max_range, sigma, height)
    # world = R_i p_i + o_i  =>  p2 = R2^T R1 p1 + R2^T (o1 - o2)
    R = R2.T @ R1
    t = R2.T @ (o1 - o2)
    zero = np.zeros(3)
    return p1.astype(np.float32), p2.astype(np.float32), R, t, zero, zero


# ----------------------------------------------------------------------------
# indoor room pair: dense, map-sized clouds
# ----------------------------------------------------------------------------


def _room(rng, W=4.0, D=3.0, H=2.2, n_furniture=40):
    prims = [
        _Rect([0, 0, 0], [W, 0, 0], [0, D, 0]),
        _Rect([0, 0, 0], [W, 0, 0], [0, 0, H]),
        _Rect([0, D, 0], [W, 0, 0], [0, 0, H]),
        _Rect([0, 0, 0], [0, D, 0], [0, 0, H]),
        _Rect([W, 0, 0], [0, D, 0], [0, 0, H]),
    ]
    for _ in range(n_furniture):
        sx, sy = rng.uniform(0.1, 0.4, 2)
        sz = rng.uniform(0.15, 0.6)
        x0 = rng.uniform(0.1, W - sx - 0.1)
        y0 = rng.uniform(0.1, D - sy - 0.1)
        prims.append(_Box([x0, y0, 0.0], [x0 + sx, y0 + sy, sz]))
        r = rng.uniform(0.02, 0.08)
        h = rng.uniform(0.15, 0.5)
        prims.append(_Cylinder([x0 + sx / 2, y0 + sy / 2, sz], r, h))
    return prims


def indoor_pair(seed: int, n: int = 2_000_000, sigma: float = 0.005, max_t: float = 2.0):
    """Two independent dense samples of one room; the target is moved by a
    uniform random rotation and a translation of at most ``max_t``.

    Returns ``(src, tgt, R, t, vp_src, vp_tgt)`` with the room centre as the
    viewpoint of each cloud.
    """
    rng = np.random.default_rng(seed)
    prims = _room(rng)
    src = _sample_region(prims, rng, n, sigma=sigma)
    tgt_w = _sample_region(prims, rng, n, sigma=sigma)
    R = random_rotation(rng)
    t = random_translation(rng, max_t)
    vp = np.array([2.0, 1.5, 1.1])
    return src.astype(np.float32), _apply(R, t, tgt_w), R, t, vp, R @ vp + t


# ----------------------------------------------------------------------------
# batches of uneven pairs and serving clouds
# ----------------------------------------------------------------------------


def batch_pairs(seed: int, n_pairs: int = 256, lo: int = 5000, hi: int = 300000,
                voxels=(0.05, 0.1, 0.3), max_t: float = 10.0):
    """Pairs of uneven sizes for batched registration.

    Each pair draws a raw size log-uniform in [lo, hi], a generator (cube scene
    or LiDAR) and a voxel size from ``voxels``; the target gets an extra
    random rigid motion (uniform rotation, translation <= ``max_t``).
    Yields dicts with keys src, tgt, R, t, vp_src, vp_tgt, voxel.
    """
    rng = np.random.default_rng(seed)
    for _ in range(n_pairs):
        size = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        sub = int(rng.integers(0, 2**31 - 1))
        v = float(voxels[int(rng.integers(0, len(voxels)))])
        if rng.random() < 0.5:
            src, tgt, R, t, vps, vpt = scene_pair(sub, n=size)
        else:
            az = max(64, int(round(size / 64 / 0.92)))
            src, tgt, R, t, vps, vpt = lidar_pair(sub, az_bins=az)
        R2 = random_rotation(rng)
        t2 = random_translation(rng, max_t)
        yield dict(src=src, tgt=_apply(R2, t2, tgt.astype(np.float64)),
                   R=R2 @ R, t=R2 @ t + t2, vp_src=vps, vp_tgt=R2 @ vpt + t2, voxel=v)


def map_cloud(seed: int, n: int):
    """A large cloud standing in for a resident map: a LiDAR scene or a room
    sampled with about ``n`` raw points.  Returns (xyz, viewpoint, kind)."""
    rng = np.random.default_rng(seed)
    if rng.random() < 0.5:
        prims = _room(rng, W=10.0, D=8.0, H=3.0)
        pts = _sample_region(prims, rng, n, sigma=0.005)
        return pts.astype(np.float32), np.array([5.0, 4.0, 1.5]), "indoor"
    az = max(256, int(round(n / 64 / 0.92)))
    src, _, _, _, vp, _ = lidar_pair(int(rng.integers(0, 2**31 - 1)), az_bins=az)
    return src, vp, "lidar"


def query_scan(seed: int, n: int):
    """A query cloud of about ``n`` raw points from the cube-scene generator."""
    src, _, _, _, vp, _ = scene_pair(seed, n=n)
    return src, vp
