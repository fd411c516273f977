"""Pins of the FP64 oracle against what the paper and mathematics fix:
closed forms, invariants, special cases that reduce to library routines, and
brute force on tiny inputs.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from synth import random_rotation, random_translation, scene_pair

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PI = math.pi


# ----------------------------------------------------------------------------
# voxelisation (input of the method, Sec. III-A)
# ----------------------------------------------------------------------------


def _voxel_by_dict(x, v):
    """Brute force: a dict keyed by the integer voxel triple, members kept in
    input order, voxels numbered in order of first appearance."""
    order, members = [], {}
    for r, p in enumerate(x):
        k = tuple(int(math.floor(float(c) / float(v))) for c in p[:3])
        if k not in members:
            members[k] = []
            order.append(k)
        members[k].append(r)
    cent, assign = [], np.zeros(len(x), np.int32)
    for o, k in enumerate(order):
        s = [0.0, 0.0, 0.0]
        for r in members[k]:
            for a in range(3):
                s[a] += float(x[r][a])
            assign[r] = o
        cent.append([np.float32(s[a] / len(members[k])) for a in range(3)])
    return np.array(cent, np.float32).reshape(-1, 3), assign


def test_voxelize_matches_dict_bruteforce(orc):
    rng = np.random.default_rng(0)
    x = rng.normal(0, 0.7, (3000, 3)).astype(np.float32)
    cent, assign = orc.voxelize(x, 0.25)
    bc, ba = _voxel_by_dict(x, np.float32(0.25))
    assert np.array_equal(assign, ba)
    assert np.array_equal(cent[:, :3], bc)
    assert np.all(cent[:, 3] == 0)


def test_voxelize_faces_and_negative_floor(orc):
    # v = 0.5 is exact in binary: x = k v lies on a face and belongs to voxel k
    # (half-open cells); -0.25 belongs to voxel -1 (floor, not truncation).
    x = np.array([[1.0, 0, 0], [1.4, 0, 0], [0.99, 0, 0], [-0.25, 0, 0], [-0.5, 0, 0], [-0.51, 0, 0]],
                 np.float32)
    cent, assign = orc.voxelize(x, 0.5)
    assert list(assign) == [0, 0, 1, 2, 2, 3]
    assert cent[0, 0] == np.float32((1.0 + np.float64(np.float32(1.4))) / 2)
    assert cent[2, 0] == np.float32((-0.25 - 0.5) / 2)


def test_voxelize_permutation_changes_order_not_set(orc):
    rng = np.random.default_rng(1)
    # coordinates on a 1/64 grid: every FP64 partial sum is exact, so centroids
    # do not depend on summation order
    x = (rng.integers(-200, 200, (2000, 3)) / 64.0).astype(np.float32)
    c1, _ = orc.voxelize(x, 0.3)
    perm = rng.permutation(len(x))
    c2, _ = orc.voxelize(x[perm], 0.3)
    s1 = sorted(map(tuple, c1.tolist()))
    s2 = sorted(map(tuple, c2.tolist()))
    assert s1 == s2


def test_voxelize_range_error(orc):
    x = np.array([[0.0, 0.0, 0.0], [2.0 ** 20 * 0.1 + 1.0, 0, 0]], np.float32)
    with pytest.raises(RuntimeError):
        orc.voxelize(x, 0.1)


# ----------------------------------------------------------------------------
# radius search (Eq. A1)
# ----------------------------------------------------------------------------


def test_radius_grid_equals_bruteforce(orc):
    rng = np.random.default_rng(2)
    p = rng.uniform(-1, 1, (1500, 3)).astype(np.float32)
    for r in (0.05, 0.2, 0.37):
        ob, nb = orc.radius_search(p, r, "brute")
        og, ng = orc.radius_search(p, r, "grid")
        assert np.array_equal(ob, og)
        assert np.array_equal(nb, ng)


def test_radius_vs_kdtree_and_symmetry(orc):
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(3)
    p = rng.uniform(0, 2, (1200, 3)).astype(np.float32)
    r = np.float32(0.2)
    offs, nbr = orc.radius_search(p, r, "brute")
    tree = cKDTree(p.astype(np.float64))
    pd = p.astype(np.float64)
    for q in range(len(p)):
        mine = set(nbr[offs[q]:offs[q + 1]].tolist())
        assert q in mine
        ref = set(tree.query_ball_point(pd[q], float(r)))
        for s in mine ^ ref:  # may differ only at the boundary
            d = np.linalg.norm(pd[s] - pd[q])
            assert abs(d - float(r)) < 1e-9
    # s in I(q)  <=>  q in I(s)
    pairs = {(q, s) for q in range(len(p)) for s in nbr[offs[q]:offs[q + 1]].tolist()}
    assert all((s, q) in pairs for (q, s) in pairs)


def test_radius_strict_boundary(orc):
    # exact distance r is outside (strict < in Eq. A1)
    p = np.array([[0, 0, 0], [0.5, 0, 0], [0, 0.25, 0]], np.float32)
    offs, nbr = orc.radius_search(p, 0.5, "brute")
    assert nbr[offs[0]:offs[1]].tolist() == [0, 2]


# ----------------------------------------------------------------------------
# eigen-decomposition and normals (Sec. III-C; Algorithm 1 step 1)
# ----------------------------------------------------------------------------


def test_jacobi_vs_lapack_and_closed_forms(orc):
    rng = np.random.default_rng(4)
    for _ in range(200):
        M = rng.normal(size=(3, 3))
        A = M @ M.T
        w, V = orc.eig3_jacobi(A)
        wl = np.linalg.eigvalsh(A)[::-1]
        assert np.allclose(w, wl, rtol=1e-12, atol=1e-13)
        assert np.allclose(A @ V, V * w, atol=1e-11)
        assert np.allclose(V.T @ V, np.eye(3), atol=1e-12)
    w, V = orc.eig3_jacobi(np.diag([0.5, 3.0, 1.0]))
    assert np.allclose(w, [3.0, 1.0, 0.5])
    assert np.allclose(np.abs(V[:, 2]), [1, 0, 0])
    R = random_rotation(rng)
    A = R @ np.diag([2.0, 0.7, 0.01]) @ R.T
    w, V = orc.eig3_jacobi(A)
    assert np.allclose(w, [2.0, 0.7, 0.01], atol=1e-13)
    assert abs(abs(V[:, 2] @ R[:, 2]) - 1) < 1e-12


def _grid_plane(n=21, h=0.1, z=0.0):
    g = np.arange(n) * h
    xx, yy = np.meshgrid(g, g)
    return np.stack([xx.ravel(), yy.ravel(), np.full(xx.size, z)], 1).astype(np.float32)


def test_normals_plane_line_and_orientation(orc):
    p = _grid_plane()
    prm = orc.OracleParams(0.1, viewpoint=[1.0, 1.0, 5.0])
    offs, nbr = orc.radius_search(p, prm.r_fpfh)
    n4, ev, flags, nn = orc.normals(p, offs, nbr, prm)
    assert np.all(flags & 1)
    assert np.allclose(n4[:, :3], [0, 0, 1], atol=1e-12)  # toward the viewpoint above
    assert np.all(ev[:, 2] == 0)
    prm_below = orc.OracleParams(0.1, viewpoint=[1.0, 1.0, -5.0])
    n4b, _, _, _ = orc.normals(p, offs, nbr, prm_below)
    assert np.allclose(n4b[:, :3], [0, 0, -1], atol=1e-12)
    # a pole: points on a line have p_lin = 1 and are rejected by tau_lin
    line = np.stack([np.arange(40) * 0.1, np.zeros(40), np.zeros(40)], 1).astype(np.float32)
    offs, nbr = orc.radius_search(line, prm.r_fpfh)
    n4, ev, flags, nn = orc.normals(line, offs, nbr, prm)
    assert np.all(flags[(nn >= 3)] & 4)
    assert not np.any(flags & 1)
    assert np.allclose(n4[nn >= 3, 3], 1.0)
    # isolated points (|I| < tau_num) never reach PCA
    iso = np.array([[0, 0, 0], [0.2, 0, 0], [5, 5, 5]], np.float32)
    offs, nbr = orc.radius_search(iso, prm.r_fpfh)
    _, _, flags, _ = orc.normals(iso, offs, nbr, prm)
    assert not np.any(flags)


def test_normals_rnormal_subsample_and_counts(orc):
    # q at the origin with 2 points inside r_normal and 3 more inside r_FPFH
    p = np.array([[0, 0, 0], [0.2, 0, 0], [0, 0.2, 0], [0.4, 0, 0], [0, 0.4, 0], [0.3, 0.3, 0]],
                 np.float32)
    prm = orc.OracleParams(0.1)  # r_normal 0.35, r_FPFH 0.5
    offs, nbr = orc.radius_search(p, prm.r_fpfh)
    _, _, flags, nn = orc.normals(p, offs, nbr, prm)
    assert nn[0] == 3 and offs[1] - offs[0] == 6
    prm4 = orc.OracleParams(0.1, tau_num=4)
    _, _, flags4, _ = orc.normals(p, offs, nbr, prm4)
    assert not (flags4[0] & 4)  # |P_normal| = 3 < 4: no PCA


def test_normals_ellipse_known_axes(orc):
    # points on an ellipse in a rotated plane: smallest axis = plane normal,
    # p_lin = (a^2 - b^2) / a^2 for semi-axes a > b (covariance diag(a^2/2, b^2/2, 0))
    rng = np.random.default_rng(5)
    R = random_rotation(rng)
    t = np.linspace(0, 2 * PI, 64, endpoint=False)
    a, b = 0.3, 0.2
    loc = np.stack([a * np.cos(t), b * np.sin(t), np.zeros_like(t)], 1)
    pts = np.concatenate([[[0, 0, 0]], loc]) @ R.T
    pts = pts.astype(np.float32)
    prm = orc.OracleParams(0.1, r_normal=0.35, r_fpfh=0.5, viewpoint=R[:, 2] * 10)
    offs, nbr = orc.radius_search(pts, prm.r_fpfh)
    n4, ev, flags, _ = orc.normals(pts, offs, nbr, prm)
    assert flags[0] & 1
    assert abs(n4[0, :3] @ R[:, 2] - 1) < 1e-6
    assert abs(n4[0, 3] - (a * a - b * b) / (a * a)) < 1e-5


# ----------------------------------------------------------------------------
# pair features (Eq. A2), bins (Eq. A3)
# ----------------------------------------------------------------------------


def test_pair_features_golden(orc):
    g = json.load(open(os.path.join(GOLDEN, "pair_features.json")))
    lo = [-PI, -1.0, -1.0]
    hi = [PI, 1.0, 1.0]
    for c in g["cases"]:
        f = orc.pair_features(c["pq"], c["nq"], c["pk"], c["nk"])
        assert f is not None, c["name"]
        assert np.allclose(f, c["f"], atol=2e-7), (c["name"], f)
        bins = [orc.feature_bin(f[l], lo[l], hi[l], g["H"]) for l in range(3)]
        assert bins == c["bins"], (c["name"], bins)


def test_pair_features_sphere_sweep(orc):
    # outward normals on a sphere of radius R: f1 = theta, f2 = 0, f3 = -c/(2R)
    rng = np.random.default_rng(6)
    for _ in range(50):
        Rs = rng.uniform(0.3, 2.0)
        th = rng.uniform(0.05, 1.5)
        Q = random_rotation(rng)
        a = Q @ np.array([1.0, 0, 0])
        b = Q @ np.array([math.cos(th), math.sin(th), 0])
        pq = (Rs * a).astype(np.float32)
        pk = (Rs * b).astype(np.float32)
        f = orc.pair_features(pq, a, pk, b)
        chord = np.linalg.norm(pk.astype(np.float64) - pq.astype(np.float64))
        assert abs(f[0] - th) < 1e-5 and abs(f[1]) < 1e-6
        assert abs(f[2] + chord / (2 * Rs)) < 1e-5
        f = orc.pair_features(pq, -a, pk, -b)
        assert abs(f[0] + th) < 1e-5 and abs(f[2] - chord / (2 * Rs)) < 1e-5


def test_pair_features_degenerate(orc):
    # d parallel to u -> |d x u| = 0 -> pair skipped; coincident points skipped
    assert orc.pair_features([0, 0, 0], [1, 0, 0], [1, 0, 0], [1, 0, 0]) is None
    assert orc.pair_features([0, 0, 0], [0, 0, 1], [0, 0, 0], [0, 0, 1]) is None


def test_bins_edges(orc):
    H = 11
    assert orc.feature_bin(-PI, -PI, PI, H) == 0
    assert orc.feature_bin(PI, -PI, PI, H) == H - 1  # upper end clamps (epsilon of Eq. A3)
    assert orc.feature_bin(1.0, -1, 1, H) == H - 1
    assert orc.feature_bin(-1.0, -1, 1, H) == 0
    for h in range(H):
        mid = -1 + (h + 0.5) * 2 / H
        assert orc.feature_bin(mid, -1, 1, H) == h


# ----------------------------------------------------------------------------
# SPFH (Eq. A4), FPFH (Eq. A5), whole chain
# ----------------------------------------------------------------------------


def test_spfh_plane_closed_form(orc):
    p = _grid_plane()
    prm = orc.OracleParams(0.1, viewpoint=[1, 1, 3])
    out = orc.faster_pfh(p, prm)
    H = 11
    rows = out["spfh"][out["flags"] & 1 > 0]
    expect = np.zeros(3 * H)
    expect[[5, H + 5, 2 * H + 5]] = 100.0
    assert np.allclose(rows, expect)


@pytest.fixture(scope="module")
def scene_fp(orc):
    src, tgt, R, t, vps, vpt = scene_pair(11, n=6000)
    vs, _ = orc.voxelize(src, 0.1)
    prm = orc.OracleParams(0.1, viewpoint=vps)
    return vs, prm, orc.faster_pfh(vs, prm)


def test_spfh_normalisation(scene_fp):
    _, _, out = scene_fp
    H = 11
    sp, npairs = out["spfh"], out["npairs"]
    has = npairs > 0
    for l in range(3):
        assert np.allclose(sp[has, l * H:(l + 1) * H].sum(1), 100.0, atol=1e-9)
    assert np.all(sp[~has] == 0)


def test_fpfh_closed_form_sum(scene_fp):
    vs, _, out = scene_fp
    H = 11
    p = vs[:, :3].astype(np.float64)
    for row, q in enumerate(out["J"]):
        ks = [k for k in out["vnbr"][out["voffs"][q]:out["voffs"][q + 1]] if k != q]
        inv = sum(1.0 / np.linalg.norm(p[k] - p[q]) for k in ks)
        for l in range(3):
            s_q = out["spfh"][q, l * H:(l + 1) * H].sum()
            s_k = [out["spfh"][k, l * H:(l + 1) * H].sum() for k in ks]
            # every neighbour third sums to 100 (or 0 if it had no pair)
            expect = s_q + sum(sk / np.linalg.norm(p[k] - p[q]) for sk, k in zip(s_k, ks)) / len(ks)
            assert abs(out["fpfh"][row, l * H:(l + 1) * H].sum() - expect) < 1e-9 * max(1, expect)
            if s_q == 100 and all(abs(sk - 100) < 1e-9 for sk in s_k):
                assert abs(out["fpfh"][row, l * H:(l + 1) * H].sum() - (100 + 100 * inv / len(ks))) < 1e-7


def test_step2_valid_filter_definition(scene_fp):
    _, prm, out = scene_fp
    B = (out["flags"] & 1) > 0
    for q in range(len(B)):
        lst = out["nbr"][out["offs"][q]:out["offs"][q + 1]]
        vl = out["vnbr"][out["voffs"][q]:out["voffs"][q + 1]]
        if B[q]:
            assert vl.tolist() == [i for i in lst.tolist() if B[i]]
        else:
            assert len(vl) == 0
        inJ = bool(out["flags"][q] & 2)
        assert inJ == (B[q] and len(vl) >= prm.tau_num)
    assert np.all(np.diff(out["J"]) > 0)


def test_descriptor_rigid_invariance(orc, scene_fp):
    """Eq. 1: a rigid motion of the voxelised cloud and of the viewpoint
    leaves neighbour sets, p_lin and descriptors unchanged except where a
    distance sits on a radius or a feature on a bin edge (FP32 rounding of
    the moved coordinates)."""
    vs, prm, out = scene_fp
    rng = np.random.default_rng(7)
    R = random_rotation(rng)
    t = random_translation(rng, 3.0)
    moved = (vs[:, :3].astype(np.float64) @ R.T + t).astype(np.float32)
    prm2 = orc.OracleParams(0.1, viewpoint=R @ prm.viewpoint + t)
    out2 = orc.faster_pfh(moved, prm2)
    same_lists = np.mean(np.diff(out["offs"]) == np.diff(out2["offs"]))
    assert same_lists > 0.999
    both = (out["flags"] & 1 > 0) & (out2["flags"] & 1 > 0)
    n_rot = out["normal4"][both, :3] @ R.T
    assert np.median(np.abs(np.sum(n_rot * out2["normal4"][both, :3], 1))) > 1 - 1e-9
    if np.array_equal(out["J"], out2["J"]):
        d = np.abs(out["fpfh"] - out2["fpfh"]).max(1)
        assert np.mean(d < 1e-6 * np.abs(out["fpfh"]).max()) > 0.9


def test_descriptor_permutation_invariance(orc, scene_fp):
    vs, prm, out = scene_fp
    rng = np.random.default_rng(8)
    perm = rng.permutation(len(vs))
    out2 = orc.faster_pfh(vs[perm], prm)
    inv = np.argsort(perm)
    # J maps through the permutation; per-point descriptors are the same set
    assert sorted(perm[out2["J"]].tolist()) == out["J"].tolist()
    row_of = {q: r for r, q in enumerate(out["J"])}
    worst = 0.0
    for r2, q2 in enumerate(out2["J"]):
        worst = max(worst, np.abs(out2["fpfh"][r2] - out["fpfh"][row_of[perm[q2]]]).max())
    assert worst < 1e-9 * np.abs(out["fpfh"]).max()
    assert inv.shape == perm.shape


# ----------------------------------------------------------------------------
# mutual matching (Sec. III-C)
# ----------------------------------------------------------------------------


def test_nearest_vs_kdtree(orc):
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(9)
    X = rng.random((700, 33)) * 50
    Y = rng.random((900, 33)) * 50
    nn, d1, d2 = orc.nearest(X, Y)
    dd, ii = cKDTree(Y).query(X, k=2)
    assert np.array_equal(nn, ii[:, 0])
    assert np.allclose(d1, dd[:, 0], rtol=1e-12)
    assert np.allclose(d2, dd[:, 1], rtol=1e-12)


def test_mutual_planted_permutation_and_transpose(orc):
    rng = np.random.default_rng(10)
    FP = rng.random((500, 33)) * 100
    perm = rng.permutation(500)
    FQ = FP[perm] + rng.normal(0, 1e-3, FP.shape)
    A, _ = orc.mutual_match(FP, FQ)
    # row i of P is row inv[i] of Q
    inv = np.argsort(perm)
    assert len(A) == 500 and np.array_equal(A["j"], inv[A["i"]])
    # random sets: partial bijection, and swapping P and Q transposes A
    FQ2 = rng.random((640, 33)) * 100
    A1, _ = orc.mutual_match(FP, FQ2)
    A2, _ = orc.mutual_match(FQ2, FP)
    assert len(set(A1["j"].tolist())) == len(A1)
    assert sorted(zip(A1["i"].tolist(), A1["j"].tolist())) == sorted(zip(A2["j"].tolist(), A2["i"].tolist()))


def test_mutual_ties_lower_index(orc):
    FP = np.array([[0.0, 0.0], [10.0, 10.0]])
    FQ = np.array([[1.0, 0.0], [0.0, 1.0], [10.0, 10.0]])  # rows 0 and 1 tie for P row 0
    A, s = orc.mutual_match(FP, FQ)
    assert s["nn_pq"][0] == 0 and s["d1p"][0] == 1.0 and s["d2p"][0] == 1.0
    assert A["i"].tolist() == [0, 1] and A["j"].tolist() == [0, 2]
