"""Downstream of matching, for the end-to-end check only (TEST INFRASTRUCTURE).

Ratio-based top-N_tau selection and k-core pruning follow Sec. III-D; the
pose comes from the GNC-TLS non-minimal solver of Sec. III-E (Yang et al.,
"Graduated Non-Convexity for Robust Spatial Perception", RA-L 2020) on top of
a weighted closed-form rigid alignment (Horn 1987 / Arun et al. 1987, SVD
form).  Success is judged as in Sec. IV-A: rotation error < 5 deg and
translation error < 2 m.
"""
from __future__ import annotations

import math

import numpy as np

from .core import load


def ratio_filter(A, n_tau=3000):
    """Keep the n_tau correspondences with the lowest descriptor distance
    ratio d1/d2 (Sec. III-D, Lowe's ratio test); ties go to the lower i.
    Returns the kept rows of A in ascending ratio."""
    if len(A) == 0:
        return A
    d2 = np.asarray(A["d2"], np.float64)
    ratio = np.where(d2 > 0, np.asarray(A["d1"], np.float64) / np.where(d2 > 0, d2, 1.0), 1.0)
    order = np.lexsort((np.asarray(A["i"]), ratio))
    return A[order[:n_tau]]


def invariant_graph(a, b, beta):
    """Compatibility graph of Sec. III-D: vertices are correspondences
    (a[k] <-> b[k]); an edge joins k and k' when the pairwise invariant of
    Eq. 3 holds, | |b_k - b_k'| - |a_k - a_k'| | <= 2 beta.
    Returns the symmetric CSR (offs int64, adj int32)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    n = len(a)
    rows = []
    for s in range(0, n, 512):
        da = np.linalg.norm(a[s:s + 512, None, :] - a[None, :, :], axis=2)
        db = np.linalg.norm(b[s:s + 512, None, :] - b[None, :, :], axis=2)
        ok = np.abs(db - da) <= 2.0 * beta
        for r in range(ok.shape[0]):
            ok[r, s + r] = False
        rows.extend(np.nonzero(row)[0].astype(np.int32) for row in ok)
    offs = np.zeros(n + 1, np.int64)
    offs[1:] = np.cumsum([len(r) for r in rows])
    adj = np.concatenate(rows) if n else np.zeros(0, np.int32)
    return offs, adj


def core_numbers(offs, adj):
    """Core number of every vertex (Batagelj & Zaversnik peeling)."""
    lib = load()
    n = len(offs) - 1
    core = np.zeros(max(n, 1), np.int32)
    if n:
        lib.orc_core_numbers(n, np.ascontiguousarray(offs, np.int64),
                             np.ascontiguousarray(adj if len(adj) else np.zeros(1, np.int32), np.int32), core)
    return core[:n]


def max_kcore(offs, adj):
    """Vertices of the maximum k-core (Sec. III-D): those whose core number
    equals the largest core number in the graph."""
    core = core_numbers(offs, adj)
    if len(core) == 0:
        return np.zeros(0, np.int64)
    return np.nonzero(core == core.max())[0]


def horn(a, b, w=None):
    """Weighted least-squares rigid motion: argmin sum w |b - R a - t|^2 over
    SO(3) x R^3 via the SVD of the weighted cross-covariance."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    w = np.ones(len(a)) if w is None else np.asarray(w, np.float64)
    sw = w.sum()
    ca = (w[:, None] * a).sum(0) / sw
    cb = (w[:, None] * b).sum(0) / sw
    H = ((a - ca) * w[:, None]).T @ (b - cb)
    U, _, Vt = np.linalg.svd(H)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(Vt.T @ U.T)) or 1.0])
    R = Vt.T @ D @ U.T
    return R, cb - R @ ca


def gnc_tls(a, b, noise_bound, max_iters=100, mu_factor=1.4, tol=1e-12):
    """GNC with the truncated-least-squares loss (Sec. III-E, Yang et al.
    2020): alternate a weighted rigid fit with the closed-form TLS weight
    update while the surrogate parameter mu grows by ``mu_factor``.
    Returns (R, t, weights)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    n = len(a)
    w = np.ones(n)
    c2 = noise_bound ** 2
    R, t = horn(a, b, w)
    r2 = np.sum((b - a @ R.T - t) ** 2, axis=1)
    rmax2 = r2.max() if n else 0.0
    if rmax2 <= c2:
        return R, t, w
    mu = c2 / max(2.0 * rmax2 - c2, 1e-30)
    prev_cost = np.inf
    for _ in range(max_iters):
        lo = mu / (mu + 1.0) * c2
        hi = (mu + 1.0) / mu * c2
        w = np.where(r2 <= lo, 1.0, np.where(r2 >= hi, 0.0,
                     math.sqrt(c2) * np.sqrt(mu * (mu + 1.0)) / np.sqrt(np.maximum(r2, 1e-300)) - mu))
        if np.count_nonzero(w > 0) < 3:
            break
        R, t = horn(a, b, w)
        r2 = np.sum((b - a @ R.T - t) ** 2, axis=1)
        cost = float(np.sum(w * r2))
        if abs(cost - prev_cost) < tol:
            break
        prev_cost = cost
        mu *= mu_factor
    return R, t, w


def register(A, src_pts, tgt_pts, voxel, n_tau=3000):
    """Correspondences -> pose: ratio filter, invariant graph, max k-core,
    GNC-TLS (Secs. III-D, III-E; beta = 1.5 v, N_tau = 3000 from Sec. IV-B).
    A has fields i (source index), j (target index), d1, d2.
    Returns (R, t, n_inliers)."""
    beta = 1.5 * voxel
    if len(A) < 3:
        return np.eye(3), np.zeros(3), 0
    sel = ratio_filter(A, n_tau)
    a = np.asarray(src_pts, np.float64)[np.asarray(sel["i"]), :3]
    b = np.asarray(tgt_pts, np.float64)[np.asarray(sel["j"]), :3]
    offs, adj = invariant_graph(a, b, beta)
    keep = max_kcore(offs, adj)
    if len(keep) < 3:
        return np.eye(3), np.zeros(3), 0
    R, t, w = gnc_tls(a[keep], b[keep], beta)
    return R, t, int((w > 0.5).sum())


def pose_errors(R_est, t_est, R_gt, t_gt):
    """Rotation error in degrees and translation error (Euclidean) in m."""
    c = (np.trace(np.asarray(R_est).T @ np.asarray(R_gt)) - 1.0) / 2.0
    rot = math.degrees(math.acos(min(1.0, max(-1.0, c))))
    return rot, float(np.linalg.norm(np.asarray(t_est) - np.asarray(t_gt)))


def is_success(R_est, t_est, R_gt, t_gt, rot_deg=5.0, trans_m=2.0):
    """Success criterion of Sec. IV-A."""
    rot, tr = pose_errors(R_est, t_est, R_gt, t_gt)
    return rot < rot_deg and tr < trans_m
