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
    when every well-posed normal may be off by up to ``eps`` rad (a scalar,
    or per point: then a pair takes the larger of its two points' values)
    and an ill-posed one by anything.  Bounds, with s = |d x u| and r the norm of
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
    if np.ndim(eps):
        e_pt = np.asarray(eps, np.float64)
        eps = np.maximum(e_pt[q], e_pt[k])
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


# ----------------------------------------------------------------------------
# chained parity: which points and pairs a band can move
# ----------------------------------------------------------------------------

NORMAL_TOL_RAD = 1e-5
LIN_BAND = 1e-5


def lin_bands(pts, f, tau_lin):
    """From the oracle's Faster-PFH chain ``f`` of one cloud: the points whose
    reliability flag B may differ at FP32 precision (p_lin within 1e-5 of
    tau_lin) and the points whose membership in J may differ (those, and
    every point with such a neighbour: |I_valid| can change).
    Returns (b_band, j_band)."""
    n = len(pts)
    n4, fl = f["normal4"], f["flags"]
    b_band = ((fl & 4) > 0) & (np.abs(n4[:, 3] - tau_lin) < LIN_BAND)
    owner = np.repeat(np.arange(n), np.diff(f["offs"]))
    j_band = b_band.copy()
    if b_band.any():
        j_band[np.unique(owner[b_band[f["nbr"]]])] = True
    return b_band, j_band


def row_allowance(pts, J, voffs, vnbr, n_marg, npairs, F):
    """Per FPFH row (rows of F, points J): the L2 norm of the deviation the
    row may show, every bin within 1e-4 at the 100-per-histogram scale plus
    the allowance of its own and its neighbours' flip-prone pairs."""
    a_fp = fpfh_allowance(pts, J, voffs, vnbr, spfh_allowance(n_marg, npairs))
    allow = np.zeros(len(F))
    for l in range(3):
        tol = BIN_TOL * np.maximum(F[:, l * H:(l + 1) * H].sum(1), 100.0) / 100.0 + a_fp
        allow += H * tol * tol
    return np.sqrt(allow)


def attribute_pairs(A_o, A_g, fo_p, fo_q, Jo_p, Jo_q, fg_p, fg_q, Jg_p, Jg_q, allow_p, allow_q, mutual_match):
    """Correspondence sets of a reference chain (A_o) and of the GPU chain
    (A_g), both with i, j as point indices; fo_* / fg_* the two chains'
    descriptors (rows in the order of Jo_* / Jg_*); allow_* the deviation a
    row of the reference's J may show (the band).  The nearest neighbours are
    taken on both descriptor sets (FP64).  Every pair in one set and not the
    other must be attributed to a band:
      - membership: an end point, or a nearest neighbour involved, is not in
        both J (the J band is checked separately);
      - band: every nearest-neighbour decision that differs between the two
        descriptor sets (row i: reference NN a, GPU NN b) is a swap that the
        rows' deviations can cause, d_o(i, b) - d_o(i, a) <=
        2 allow_i + allow_a + allow_b (triangle inequality).
    A differing pair whose decisions all agree, or a swap beyond the band,
    is unexplained.  Pass the measured deviations |fg - fo| of the rows as
    allow_* after checking them against the allowed ones, so that a swap is
    explained by the deviations that actually occurred.
    Returns (unexplained pairs, counts per reason)."""
    idx = lambda J: {int(q): r for r, q in enumerate(J)}
    ro_p, ro_q, rg_p, rg_q = idx(Jo_p), idx(Jo_q), idx(Jg_p), idx(Jg_q)
    _, so = mutual_match(fo_p, fo_q)
    _, sg = mutual_match(fg_p, fg_q)
    nn_o_pq = lambda i: int(Jo_q[so["nn_pq"][ro_p[i]]])
    nn_g_pq = lambda i: int(Jg_q[sg["nn_pq"][rg_p[i]]])
    nn_o_qp = lambda j: int(Jo_p[so["nn_qp"][ro_q[j]]])
    nn_g_qp = lambda j: int(Jg_p[sg["nn_qp"][rg_q[j]]])
    d_o = lambda i, j: float(np.linalg.norm(fo_p[ro_p[i]] - fo_q[ro_q[j]]))
    both_p = lambda i: i in ro_p and i in rg_p
    both_q = lambda j: j in ro_q and j in rg_q

    def row_ok(i):  # None: membership; True / False: agree or in band / beyond band
        if not both_p(i):
            return None
        a, b = nn_o_pq(i), nn_g_pq(i)
        if a == b:
            return True
        if not (both_q(a) and both_q(b)):
            return None
        lim = 2 * allow_p[ro_p[i]] + allow_q[ro_q[a]] + allow_q[ro_q[b]]
        return "swap" if d_o(i, b) - d_o(i, a) <= lim * (1 + 1e-9) + 1e-9 else False

    def col_ok(j):
        if not both_q(j):
            return None
        a, b = nn_o_qp(j), nn_g_qp(j)
        if a == b:
            return True
        if not (both_p(a) and both_p(b)):
            return None
        lim = 2 * allow_q[ro_q[j]] + allow_p[ro_p[a]] + allow_p[ro_p[b]]
        return "swap" if d_o(a, j) - d_o(b, j) >= -lim * (1 + 1e-9) - 1e-9 else False

    ref = set(zip(A_o["i"].tolist(), A_o["j"].tolist()))
    got = set(zip(A_g["i"].tolist(), A_g["j"].tolist()))
    reasons = dict(membership=0, band=0)
    unexplained = []
    for i, j in sorted(ref ^ got):
        cols = {j}
        if both_p(i):
            cols |= {nn_o_pq(i), nn_g_pq(i)}
        checks = [row_ok(i)] + [col_ok(c) for c in sorted(cols)]
        if any(c is False for c in checks):
            unexplained.append((i, j))
        elif any(c is None for c in checks):
            reasons["membership"] += 1
        elif any(c == "swap" for c in checks):
            reasons["band"] += 1
        else:
            unexplained.append((i, j))  # every decision agrees: the sets should too
    reasons["differing"] = len(ref ^ got)
    reasons["pairs"] = len(ref)
    return unexplained, reasons
