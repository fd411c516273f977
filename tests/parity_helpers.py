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
