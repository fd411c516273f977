"""Pins of the oracle's classic FPFH (the baseline of Sec. III-C, Fig. 2(a)):
three radius searches and no reliability filtering.  CPU only.

What fixes it: where Faster-PFH filters nothing (every point reliable), the two
methods compute the same descriptors, so classic must equal the pinned
Faster-PFH oracle bit for bit; on a plane the descriptor has a closed form;
points on a line, which Faster-PFH rejects by linearity, are kept; the point
set is exactly the brute-force set of points with three or more points within
r_normal."""
import numpy as np

from synth import scene_pair

H = 11


def _surface(n=24, h=0.1, seed=0):
    """A gently curved, noisy height field sampled on a square lattice: every
    point has dozens of neighbours within r_normal and p_lin well below 0.99."""
    rng = np.random.default_rng(seed)
    g = np.arange(n) * h
    xx, yy = np.meshgrid(g, g)
    zz = 0.15 * np.sin(xx) * np.cos(0.7 * yy) + rng.normal(0, 0.003, xx.shape)
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(np.float32)


def _brute_counts(p, r):
    x = p[:, :3].astype(np.float64)
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    return d2, (d2 < np.float64(np.float32(r)) ** 2)


def test_classic_equals_fasterpfh_where_nothing_is_filtered(orc):
    p = _surface()
    prm = orc.OracleParams(0.1, viewpoint=[1.0, 1.0, 4.0])
    f = orc.faster_pfh(p, prm)
    c = orc.classic_fpfh(p, prm)
    n = len(p)
    # precondition: Faster-PFH keeps every point
    assert len(f["J"]) == n and np.all(f["flags"] & 1)
    assert np.array_equal(c["J"], np.arange(n))
    assert np.array_equal(c["normal4"], f["normal4"])
    assert np.array_equal(c["spfh"], f["spfh"])
    assert np.array_equal(c["fpfh"], f["fpfh"])


def test_classic_point_set_and_linear_points(orc):
    g = np.arange(21) * 0.1
    xx, yy = np.meshgrid(g, g)
    plane = np.stack([xx.ravel(), yy.ravel(), np.zeros(xx.size)], 1)
    pole = np.stack([np.full(12, 6.0), np.full(12, 6.0), np.arange(12) * 0.1], 1)
    pair = np.array([[-5.0, -5.0, 0.0], [-5.2, -5.0, 0.0]])  # |P_normal| = 2: no normal
    # a star: the centre has a normal (3 points within r_normal) but no
    # neighbour with one, so it has no valid neighbour and is still described
    star = np.array([[-8.0, -8.0, 0.0], [-7.7, -8.0, 0.0], [-8.0, -7.7, 0.0]])
    p = np.concatenate([plane, pole, pair, star]).astype(np.float32)
    prm = orc.OracleParams(0.1, viewpoint=[1.0, 1.0, 5.0])
    c = orc.classic_fpfh(p, prm)
    f = orc.faster_pfh(p, prm)
    _, inN = _brute_counts(p, prm.r_normal)
    expect = np.nonzero(inN.sum(1) >= 3)[0]
    assert np.array_equal(c["J"], expect)
    pole_idx = np.arange(len(plane), len(plane) + len(pole))
    assert np.all(np.isin(pole_idx, c["J"]))          # kept by classic FPFH
    assert not np.any(np.isin(pole_idx, f["J"]))      # rejected by tau_lin in Faster-PFH
    assert np.allclose(c["normal4"][pole_idx, 3], 1.0)  # p_lin of a line
    n0 = len(plane) + len(pole)
    assert not np.any(np.isin([n0, n0 + 1, n0 + 3, n0 + 4], c["J"]))
    assert n0 + 2 in c["J"] and c["npairs"][n0 + 2] == 0
    assert np.all(c["fpfh"][np.isin(c["J"], pole_idx)].sum(1) > 0)
    assert np.all(c["fpfh"][np.searchsorted(c["J"], n0 + 2)] == 0)


def test_classic_plane_closed_form(orc):
    """Exact plane, normals toward a viewpoint above: every pair has f = 0, so
    each third of SPFH is 100 in bin 5 and each third of FPFH sums to
    100 + (100/m) sum_k 1/w_k over the m neighbours within r_FPFH (third
    search), all in bin 5; the pair count is the brute-force r_FPFH count."""
    g = np.arange(15) * 0.1
    xx, yy = np.meshgrid(g, g)
    p = np.stack([xx.ravel(), yy.ravel(), np.zeros(xx.size)], 1).astype(np.float32)
    prm = orc.OracleParams(0.1, viewpoint=[0.7, 0.7, 3.0])
    c = orc.classic_fpfh(p, prm)
    assert np.array_equal(c["J"], np.arange(len(p)))
    d2, inF = _brute_counts(p, prm.r_fpfh)
    np.fill_diagonal(inF, False)
    m = inF.sum(1)
    assert np.array_equal(c["npairs"], m)
    inv = np.where(inF, 1.0 / np.sqrt(np.where(inF, d2, 1.0)), 0.0).sum(1)
    for l in range(3):
        third = c["fpfh"][:, l * H:(l + 1) * H]
        assert np.allclose(third[:, 5], 100.0 + 100.0 * inv / m, rtol=1e-12)
        assert np.all(np.delete(third, 5, axis=1) == 0)


def test_classic_grid_search_equals_bruteforce(orc):
    src = scene_pair(21, n=3000)[0]
    vs, _ = orc.voxelize(src, 0.1)
    prm = orc.OracleParams(0.1, viewpoint=[0.0, 0.0, 0.0])
    a = orc.classic_fpfh(vs, prm, search="grid")
    b = orc.classic_fpfh(vs, prm, search="brute")
    assert np.array_equal(a["J"], b["J"]) and np.array_equal(a["fpfh"], b["fpfh"])
    # classic FPFH describes at least every point Faster-PFH describes
    f = orc.faster_pfh(vs, prm)
    assert np.all(np.isin(f["J"], a["J"])) and len(a["J"]) > len(f["J"])
