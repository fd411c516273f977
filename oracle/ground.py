"""Geometric suppression (Sec. III-B) for the oracle: ground removal before
the descriptors (TEST INFRASTRUCTURE ONLY).

The paper removes repetitive planar structure (the ground) before feature
extraction and uses Patchwork (Lim et al., RA-L 2021) for it, a method it
does not restate.  This is the stand-in both sides implement: Patchwork's
concentric zone model and region-wise ground plane fitting, with the plane
fitted as a height field and every decision made on exact integers or on a
fixed sequence of IEEE FP64 operations, so that the CUDA path can reproduce
it bit for bit.

Per point (sensor frame, z up):
  * bin: the zone z with R_z^2 <= x^2 + y^2 < R_{z+1}^2 (and |z| < z_limit),
    the ring floor(((r - R_z) * rings_z) / (R_{z+1} - R_z)) with r the
    correctly rounded square root, the sector floor(p * sectors_z / 4) of the
    pseudo-angle p in [0, 4) (both clamped to the last index);
  * quantised coordinates rint(x * 2^quant_log2) as integers.
Per bin with min_points <= m <= max_bin_points members:
  1. lowest point representative: the sum of the k = min(n_lpr, m) lowest
     quantised heights (ties by point index); seeds are the members with
     zq * k < sum + rint(th_seeds * Q) * k;
  2. plane z = a x + b y + c by least squares over the seeds: integer moments,
     centred exactly (n S_xx - S_x S_x ...), converted once to FP64, Cramer's
     rule;
  3. n_iter times: members within th_dist of the plane
     (e^2 < th^2 (1 + a^2 + b^2), e = ((a x + b y) + c) - z, quantised units)
     are refitted (a fit of fewer than 3 points or a singular system keeps
     the previous plane and stops); the final plane classifies again;
  4. the bin is ground when a^2 + b^2 <= max_slope^2 (uprightness) and the
     mean quantised height of its ground members is below
     rint(max_ground_z * Q) (elevation); those members are removed.
Bin status: 0 too few / too many members, 1 no fit, 2 too steep, 3 too high,
4 ground.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class GroundParams:
    """Defaults: Patchwork's four-zone model (zone edges in m, rings and
    sectors per zone) and R-GPF settings; a sensor about 1.7 m above the road
    (the ground lies below -0.8 m in the sensor frame)."""

    zone_r: tuple = (2.7, 12.3, 22.1, 41.1, 80.0)
    zone_rings: tuple = (2, 4, 4, 4)
    zone_sectors: tuple = (16, 32, 54, 32)
    quant_log2: int = 8
    z_limit: float = 80.0
    n_lpr: int = 20
    th_seeds: float = 0.125
    th_dist: float = 0.125
    n_iter: int = 3
    max_slope: float = 1.0
    max_ground_z: float = -0.8
    min_points: int = 10
    max_bin_points: int = 65536


def _f(x):
    """A parameter as the FP32 value the CUDA path receives, widened."""
    return float(np.float32(x))


def n_bins(prm: GroundParams) -> int:
    return int(sum(r * s for r, s in zip(prm.zone_rings, prm.zone_sectors)))


def pseudo_angle(x, y):
    """Monotone stand-in for atan2 on [0, 4): quadrant + |y| / (|x| + |y|)
    measured from the positive x axis, counter-clockwise; exact IEEE
    operations only (no transcendental whose last bit may differ)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    p = np.zeros(x.shape)
    q0 = (y >= 0) & (x >= 0)
    q1 = (y >= 0) & (x < 0)
    q2 = (y < 0) & (x < 0)
    q3 = (y < 0) & (x >= 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        p[q0] = y[q0] / (x[q0] + y[q0])
        p[q1] = 1.0 - x[q1] / (y[q1] - x[q1])
        p[q2] = 2.0 - y[q2] / (-x[q2] - y[q2])
        p[q3] = 3.0 + x[q3] / (x[q3] - y[q3])
    return p


def ground_bins(xyz, prm: GroundParams):
    """Bin of every point (-1: outside the zones or |z| >= z_limit)."""
    p = np.asarray(xyz, np.float32)
    x = p[:, 0].astype(np.float64)
    y = p[:, 1].astype(np.float64)
    z = p[:, 2].astype(np.float64)
    r2 = x * x + y * y
    b = np.full(len(p), -1, np.int64)
    inz_all = np.abs(z) < _f(prm.z_limit)
    off = 0
    for k in range(4):
        R0, R1 = _f(prm.zone_r[k]), _f(prm.zone_r[k + 1])
        rings, sect = int(prm.zone_rings[k]), int(prm.zone_sectors[k])
        inz = inz_all & (r2 >= R0 * R0) & (r2 < R1 * R1)
        r = np.sqrt(r2[inz])
        ring = np.minimum(np.floor(((r - R0) * rings) / (R1 - R0)), rings - 1).astype(np.int64)
        sec = np.minimum(np.floor(pseudo_angle(x[inz], y[inz]) * sect / 4.0), sect - 1).astype(np.int64)
        b[inz] = off + ring * sect + sec
        off += rings * sect
    return b


def quantise(xyz, prm: GroundParams):
    Q = float(2 ** prm.quant_log2)
    return np.rint(np.asarray(xyz, np.float32)[:, :3].astype(np.float64) * Q).astype(np.int64)


def fit_plane(xq, yq, zq):
    """Least-squares height field z = a x + b y + c over integer points:
    exact integer moments, centred exactly, then FP64 Cramer's rule.  None
    for fewer than 3 points or a singular system."""
    n = len(xq)
    if n < 3:
        return None
    Sx, Sy, Sz = int(np.sum(xq)), int(np.sum(yq)), int(np.sum(zq))
    Sxx, Sxy, Syy = int(np.sum(xq * xq)), int(np.sum(xq * yq)), int(np.sum(yq * yq))
    Sxz, Syz = int(np.sum(xq * zq)), int(np.sum(yq * zq))
    cxx = float(n * Sxx - Sx * Sx)
    cxy = float(n * Sxy - Sx * Sy)
    cyy = float(n * Syy - Sy * Sy)
    cxz = float(n * Sxz - Sx * Sz)
    cyz = float(n * Syz - Sy * Sz)
    det = cxx * cyy - cxy * cxy
    if not det > 0.0:
        return None
    a = (cxz * cyy - cyz * cxy) / det
    b = (cyz * cxx - cxz * cxy) / det
    c = ((float(Sz) - a * float(Sx)) - b * float(Sy)) / float(n)
    return a, b, c


def classify(plane, xq, yq, zq, th_q):
    """Members within th_q (quantised units) of the plane, orthogonally."""
    a, b, c = plane
    e = ((a * xq.astype(np.float64) + b * yq.astype(np.float64)) + c) - zq.astype(np.float64)
    return e * e < (th_q * th_q) * ((1.0 + a * a) + b * b)


def suppress_ground(xyz, prm: GroundParams | None = None):
    """Returns dict(ground [n] bool, bins [n], planes [n_bins, 4] float64 =
    (a, b, c, status), kept = xyz[~ground])."""
    prm = prm or GroundParams()
    xyz = np.asarray(xyz, np.float32)
    n = len(xyz)
    nb = n_bins(prm)
    b = ground_bins(xyz, prm) if n else np.zeros(0, np.int64)
    q = quantise(xyz, prm) if n else np.zeros((0, 3), np.int64)
    Q = float(2 ** prm.quant_log2)
    ths = int(np.rint(_f(prm.th_seeds) * Q))
    thd = _f(prm.th_dist) * Q
    mz = int(np.rint(_f(prm.max_ground_z) * Q))
    slope2 = _f(prm.max_slope) * _f(prm.max_slope)
    ground = np.zeros(n, bool)
    planes = np.zeros((nb, 4))
    order = np.argsort(b, kind="stable")
    bs = b[order]
    starts = np.searchsorted(bs, np.arange(nb))
    ends = np.searchsorted(bs, np.arange(nb), side="right")
    for k in range(nb):
        idx = order[starts[k]:ends[k]]
        m = len(idx)
        if m < prm.min_points or m > prm.max_bin_points:
            continue  # status 0
        xq, yq, zq = q[idx, 0], q[idx, 1], q[idx, 2]
        low = np.lexsort((idx, zq))[: min(prm.n_lpr, m)]
        kk = len(low)
        lpr = int(np.sum(zq[low]))
        seeds = zq * kk < lpr + ths * kk
        plane = fit_plane(xq[seeds], yq[seeds], zq[seeds])
        if plane is None:
            planes[k, 3] = 1
            continue
        for _ in range(prm.n_iter):
            g = classify(plane, xq, yq, zq, thd)
            p2 = fit_plane(xq[g], yq[g], zq[g])
            if p2 is None:
                break
            plane = p2
        g = classify(plane, xq, yq, zq, thd)
        a, bb, c = plane
        planes[k, :3] = plane
        if not (a * a + bb * bb <= slope2):
            planes[k, 3] = 2
            continue
        ng = int(g.sum())
        if ng == 0 or not (int(np.sum(zq[g])) < mz * ng):
            planes[k, 3] = 3
            continue
        planes[k, 3] = 4
        ground[idx[g]] = True
    return dict(ground=ground, bins=b, planes=planes, kept=xyz[~ground])

