"""Pins of the oracle's geometric suppression stand-in (Sec. III-B, ground
removal by region-wise plane fitting on a concentric zone model).  CPU only.

What fixes it: a noise-free flat ground gives the exact plane (a = b = 0,
c = the quantised height) and exactly the points within th_dist; the fit
equals numpy's least squares on the same points; a tilted road is kept as
ground, a steep slope and an elevated flat roof are rejected by the
uprightness and elevation tests; low outliers do not pull the plane; the
bins partition the annulus by radius and by angle (checked against atan2);
and on a LiDAR scan pair the suppression turns a failed registration into a
successful one, the reason the paper gives for it."""
import math

import numpy as np
import pytest

from oracle import ground as G

Q = 256.0


def _disc(rmax=30.0, step=0.3, z=-1.73, f=None):
    g = np.arange(-rmax, rmax, step)
    xx, yy = np.meshgrid(g, g)
    x, y = xx.ravel(), yy.ravel()
    keep = (x * x + y * y >= 2.8 ** 2) & (x * x + y * y < (rmax - 0.5) ** 2)
    x, y = x[keep], y[keep]
    zz = np.full(x.shape, z) if f is None else f(x, y)
    return np.stack([x, y, zz], 1).astype(np.float32)


def test_flat_ground_exact_plane_and_objects():
    ground = _disc()
    # the walls of a box at (8, 5) from 0.28 m above the ground up to z = +1
    # (all farther than th_dist from the ground plane)
    t = np.linspace(0, 1, 40)
    zs = np.linspace(-1.45, 1.0, 30)
    walls = []
    for zc in zs:
        walls.append(np.stack([8 + 2 * t, np.full_like(t, 5.0), np.full_like(t, zc)], 1))
        walls.append(np.stack([np.full_like(t, 8.0), 5 + 2 * t, np.full_like(t, zc)], 1))
    walls = np.concatenate(walls).astype(np.float32)
    pts = np.concatenate([ground, walls])
    out = G.suppress_ground(pts)
    zq0 = int(np.rint(np.float64(np.float32(-1.73)) * Q))
    used = out["planes"][:, 3] == 4
    assert used.sum() > 50
    # bins without wall points: the exact plane; the wall points within
    # th_seeds of the lowest points enter the seeds of their bins, and the
    # refits move those planes back toward the ground
    clean = used.copy()
    clean[np.unique(out["bins"][len(ground):][out["bins"][len(ground):] >= 0])] = False
    assert clean.sum() > 50
    assert np.all(out["planes"][clean, 0] == 0.0) and np.all(out["planes"][clean, 1] == 0.0)
    assert np.all(out["planes"][clean, 2] == zq0)
    # every ground point removed, every wall point kept
    assert np.all(out["ground"][: len(ground)])
    assert not np.any(out["ground"][len(ground):])
    assert np.array_equal(out["kept"], walls)


def test_fit_equals_lstsq_and_tilted_road_kept():
    # the fit on scattered (not lattice-symmetric) noisy points vs LAPACK
    rng = np.random.default_rng(9)
    xy = rng.uniform([3, -2], [15, 9], (500, 2))
    zz = 0.03 * xy[:, 0] - 0.07 * xy[:, 1] - 1.5 + rng.normal(0, 0.02, 500)
    sc = np.concatenate([xy, zz[:, None]], 1).astype(np.float32)
    q = G.quantise(sc, G.GroundParams())
    a, b, c = G.fit_plane(q[:, 0], q[:, 1], q[:, 2])
    A = np.stack([q[:, 0], q[:, 1], np.ones(len(q))], 1).astype(np.float64)
    ref = np.linalg.lstsq(A, q[:, 2].astype(np.float64), rcond=None)[0]
    assert np.allclose([a, b, c], ref, rtol=1e-9, atol=1e-6)
    assert G.fit_plane(q[:2, 0], q[:2, 1], q[:2, 2]) is None
    line = np.stack([np.arange(10), 2 * np.arange(10), np.arange(10)], 1)
    assert G.fit_plane(line[:, 0], line[:, 1], line[:, 2]) is None  # collinear: singular
    f = lambda x, y: 0.015 * x - 0.01 * y - 1.8
    pts = _disc(f=f)
    out = G.suppress_ground(pts)
    assert out["ground"].all()
    used = out["planes"][:, 3] == 4
    assert np.all(np.abs(out["planes"][used, 0] - 0.015) < 2e-3)
    # the same road rising above max_ground_z is rejected where it does
    hi = G.suppress_ground(_disc(f=lambda x, y: 0.08 * x - 1.6))
    st = hi["planes"][:, 3]
    assert np.any(st == 3) and np.any(st == 4)


def test_steep_slope_and_elevated_roof_rejected():
    for f in (lambda x, y: 1.5 * x - 1.7, lambda x, y: 1.5 * y - 1.7):
        out = G.suppress_ground(_disc(f=f))
        st = out["planes"][:, 3]
        # too steep, or (seeds on one lattice line) no fit at all
        assert not out["ground"].any() and np.all(np.isin(st[st > 0], (1, 2))) and np.sum(st == 2) > 100
    roof = _disc(z=0.5)
    out = G.suppress_ground(roof)
    st = out["planes"][:, 3]
    assert not out["ground"].any() and np.all(st[st > 0] == 3)


def test_distance_is_orthogonal_to_the_plane():
    """On a 35-degree slope (accepted: uprightness limit 45 degrees) points
    0.14 m above the plane vertically are 0.115 m from it orthogonally, so
    they are ground at th_dist = 0.125 m."""
    g = np.arange(4.0, 6.0, 0.05)
    h = np.arange(0.2, 0.8, 0.05)
    xx, yy = np.meshgrid(g, h)
    x, y = xx.ravel(), yy.ravel()
    slope = np.stack([x, y, 0.7 * (x - 5.0) - 1.7], 1)
    up = slope[::25] + [0.0, 0.0, 0.14]
    pts = np.concatenate([slope, up]).astype(np.float32)
    out = G.suppress_ground(pts)
    used = np.nonzero(out["planes"][:, 3] == 4)[0]
    assert len(used) == 1 and abs(out["planes"][used[0], 0] - 0.7) < 0.01
    assert out["ground"].all()


def test_seeds_stay_below_a_low_platform():
    """A platform 0.2 m above the ground covering most of a bin: seeds are
    taken within th_seeds (0.125 m) of the lowest points, so the plane is the
    ground's exactly and the platform stays."""
    pts = _disc()
    b = G.ground_bins(pts, G.GroundParams())
    k = np.bincount(b[b >= 0]).argmax()
    members = pts[b == k]
    plat = np.concatenate([members + [0.05, 0.05, 0.2], members + [0.1, 0.1, 0.2], members + [0.15, 0.0, 0.2]])
    out = G.suppress_ground(np.concatenate([pts, plat.astype(np.float32)]))
    assert out["planes"][k, 3] == 4
    assert out["planes"][k, :3].tolist() == [0.0, 0.0, float(np.rint(np.float64(np.float32(-1.73)) * Q))]
    assert not out["ground"][len(pts):].any()


def test_min_points_per_bin():
    # a lone patch of ground points in one bin: 9 are too few, 10 are fitted
    base = np.array([[5.0 + 0.1 * i, 0.3 + 0.1 * (i % 3), -1.73 + 0.01 * (i % 2)] for i in range(10)], np.float32)
    assert not G.suppress_ground(base[:9])["ground"].any()
    assert G.suppress_ground(base)["ground"].all()


def test_low_outliers_do_not_pull_the_plane():
    pts = _disc()
    b = G.ground_bins(pts, G.GroundParams())
    k = np.bincount(b[b >= 0]).argmax()
    members = np.nonzero(b == k)[0]
    low = pts[members[:2]].copy()
    low[:, 2] = -2.5  # 0.77 m below the ground, two of the 20 lowest
    out = G.suppress_ground(np.concatenate([pts, low]))
    assert out["planes"][k, 3] == 4
    assert out["planes"][k, 0] == 0.0 and out["planes"][k, 1] == 0.0
    assert out["planes"][k, 2] == int(np.rint(np.float64(np.float32(-1.73)) * Q))
    assert not out["ground"][-2:].any() and out["ground"][: len(pts)].all()


def test_bins_partition_by_radius_and_angle():
    rng = np.random.default_rng(3)
    r = rng.uniform(0, 90, 20000)
    th = rng.uniform(-math.pi, math.pi, 20000)
    z = rng.uniform(-100, 100, 20000)
    pts = np.stack([r * np.cos(th), r * np.sin(th), z], 1).astype(np.float32)
    prm = G.GroundParams()
    b = G.ground_bins(pts, prm)
    x, y = pts[:, 0].astype(np.float64), pts[:, 1].astype(np.float64)
    rr = np.hypot(x, y)
    inside = (rr >= 2.7 + 1e-4) & (rr < 80.0 - 1e-4) & (np.abs(pts[:, 2]) < 80.0)
    outside = (rr < 2.7 - 1e-4) | (rr >= 80.0 + 1e-4) | (np.abs(pts[:, 2]) >= 80.0 + 1e-4)
    assert np.all(b[inside] >= 0) and np.all(b[outside] == -1)
    assert b.max() < G.n_bins(prm)
    # the pseudo-angle is monotone in the true angle, so a sector is an arc
    ang = np.mod(np.arctan2(y, x), 2 * math.pi)
    p = G.pseudo_angle(x, y)
    o = np.argsort(ang)
    assert np.all(np.diff(p[o]) >= 0)
    # zone and ring follow the radius (equal-width rings per zone), away from
    # ring edges
    offs = np.cumsum([0] + [r_ * s for r_, s in zip(prm.zone_rings, prm.zone_sectors)])
    bi, ri = b[inside], rr[inside]
    zone = np.searchsorted(offs, bi, side="right") - 1
    assert np.all(zone == np.searchsorted(prm.zone_r, ri, side="right") - 1)
    R = np.asarray(prm.zone_r)
    rings = np.asarray(prm.zone_rings)[zone]
    u = (ri - R[zone]) / (R[zone + 1] - R[zone]) * rings
    far = np.abs(u - np.rint(u)) > 1e-4
    ring = (bi - offs[zone]) // np.asarray(prm.zone_sectors)[zone]
    assert np.array_equal(ring[far], np.floor(u[far]).astype(np.int64))


@pytest.mark.slow
def test_suppression_lets_the_lidar_pair_register():
    import oracle
    from synth import lidar_pair

    src, tgt, R, t, vps, vpt = lidar_pair(1000, az_bins=1024)
    res = {}
    for name, (S, T) in (("plain", (src, tgt)),
                         ("suppressed", (G.suppress_ground(src)["kept"], G.suppress_ground(tgt)["kept"]))):
        A, fs, ft, vs, vt = oracle.front_end(S, T, 0.3, np.float32(vps).astype(np.float64),
                                             np.float32(vpt).astype(np.float64))
        Ro, to, _ = oracle.register(A, vs, vt, 0.3)
        res[name] = oracle.is_success(Ro, to, R, t)
    assert res["suppressed"] and not res["plain"]
