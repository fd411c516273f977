"""Tolerance helpers shared by the GPU parity tests.

Histogram bins are compared at 1e-4 on the 100-per-sub-histogram scale
(1e-4 * S_l / 100 for a sub-histogram whose oracle sum is S_l).  A pair
feature within FEATURE_BAND of a decision FP32 rounding can flip (bin edge,
atan2 cut, source choice, degenerate-pair threshold; counted per point by the
oracle) may move one count; the allowances below are the largest change such
flips can make, carried through Eq. A4 and Eq. A5.
"""
import numpy as np

H = 11
BIN_TOL = 1e-4
FEATURE_BAND = 2e-6


def hist_violation(got, ref, allowance=None):
    """Per-row max of |got - ref| / (BIN_TOL * S_l / 100 + allowance)."""
    viol = np.zeros(len(ref))
    extra = np.zeros(len(ref)) if allowance is None else allowance
    for l in range(3):
        sl = ref[:, l * H:(l + 1) * H]
        tol = BIN_TOL * np.maximum(sl.sum(1), 100.0) / 100.0 + extra
        err = np.abs(got[:, l * H:(l + 1) * H] - sl).max(1)
        viol = np.maximum(viol, err / tol)
    return viol


def spfh_allowance(n_marg, npairs):
    """2 * 100 / c per flip-prone pair of a point with c contributing pairs."""
    a = np.zeros(len(n_marg))
    ok = npairs > 0
    a[ok] = 2.0 * n_marg[ok] * 100.0 / npairs[ok]
    return a


def fpfh_allowance(pts, J, voffs, vnbr, a_sp):
    """SPFH(q)'s allowance plus (1/m) sum_k a_k / w_k over its neighbours."""
    p = pts[:, :3].astype(np.float64)
    cnt = np.diff(voffs)
    owner = np.repeat(np.arange(len(cnt)), cnt)
    k = np.asarray(vnbr, np.int64)
    keep = k != owner
    owner, k = owner[keep], k[keep]
    w = 1.0 / np.linalg.norm(p[k] - p[owner], axis=1)
    m = np.bincount(owner, minlength=len(cnt))
    s = np.bincount(owner, weights=w * a_sp[k], minlength=len(cnt))
    return (a_sp + np.where(m > 0, s / np.maximum(m, 1), 0.0))[J]


def _edge_distance(f, lo, hi):
    """Distance (f units) from f to the nearest interior bin edge of Eq. A3."""
    t = H * (f - lo) / (hi - lo)
    e = np.clip(np.rint(t), 1, H - 1)
    return np.abs(t - e) * (hi - lo) / H


def chained_pair_prone(pts, normal4, has_normal, ill, voffs, vnbr, eps, band=FEATURE_BAND):
    """Per point, the number of its SPFH pairs (Eq. A2) whose bins can change
    when every well-posed normal may be off by up to ``eps`` rad (and an
    ill-posed one by anything).  Bounds, with s = |d x u| and r the norm of
    the atan2 arguments: |df3| <= 2 eps, |df2| <= 2 eps / s + 2 eps,
    |df1| <= (2 |df2| + 2 eps) / r.  A pair is counted when a feature lies
    within its bound (+ band) of a bin edge or the atan2 cut, when the source
    choice |n_q . d| vs |n_k . d| is within 4 eps, when s or r is below 1e-3,
    or when either normal is ill-posed.  Computed from the oracle's normals."""
    p = pts[:, :3].astype(np.float64)
    cnt = np.diff(voffs)
    owner = np.repeat(np.arange(len(cnt)), cnt)
    k = np.asarray(vnbr, np.int64)
    keep = (k != owner) & has_normal[owner] & has_normal[k]
    q, k = owner[keep], k[keep]
    d = p[k] - p[q]
    dn = np.linalg.norm(d, axis=1)
    ok = dn > 0
    q, k, d, dn = q[ok], k[ok], d[ok], dn[ok]
    d0 = d / dn[:, None]
    nq, nk = normal4[q, :3], normal4[k, :3]
    cq = np.abs(np.sum(nq * d0, 1))
    ck = np.abs(np.sum(nk * d0, 1))
    swap = ~(cq >= ck)
    u = np.where(swap[:, None], nk, nq)
    nb = np.where(swap[:, None], nq, nk)
    dd = np.where(swap[:, None], -d0, d0)
    c = np.cross(dd, u)
    s = np.linalg.norm(c, axis=1)
    v = c / np.maximum(s, 1e-300)[:, None]
    w = np.cross(u, v)
    x, y = np.sum(u * nb, 1), np.sum(w * nb, 1)
    r = np.hypot(x, y)
    f1, f2, f3 = np.arctan2(y, x), np.sum(v * nb, 1), np.sum(u * dd, 1)
    b3 = 2 * eps
    b2 = 2 * eps / np.maximum(s, 1e-300) + 2 * eps
    b1 = (2 * b2 + 2 * eps) / np.maximum(r, 1e-300)
    prone = (np.abs(cq - ck) <= 4 * eps) | (s < 1e-3) | (r < 1e-3) | ill[q] | ill[k]
    prone |= _edge_distance(f1, -np.pi, np.pi) < b1 + band
    prone |= (np.pi - np.abs(f1)) < b1 + band
    prone |= _edge_distance(f2, -1.0, 1.0) < b2 + band
    prone |= _edge_distance(f3, -1.0, 1.0) < b3 + band
    return np.bincount(q, weights=prone.astype(np.float64), minlength=len(cnt)).astype(np.int64)
