"""Pins of the oracle's downstream parts (Secs. III-D, III-E) used by the
end-to-end check: rigid fit, k-core, GNC-TLS.  CPU only."""
import numpy as np
import pytest

from synth import random_rotation, random_translation, scene_pair


def test_horn_exact_without_outliers(orc):
    rng = np.random.default_rng(0)
    a = rng.normal(size=(50, 3))
    R = random_rotation(rng)
    t = random_translation(rng, 5)
    b = a @ R.T + t
    Re, te = orc.horn(a, b)
    assert np.allclose(Re, R, atol=1e-12) and np.allclose(te, t, atol=1e-12)


def test_core_numbers_vs_networkx(orc):
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(1)
    for trial in range(5):
        n = 60
        G = nx.gnp_random_graph(n, 0.1 + 0.05 * trial, seed=trial)
        offs = np.zeros(n + 1, np.int64)
        adj = []
        for v in range(n):
            nb = sorted(G.neighbors(v))
            adj.extend(nb)
            offs[v + 1] = offs[v] + len(nb)
        core = orc.core_numbers(offs, np.array(adj, np.int32))
        ref = nx.core_number(G)
        assert [ref[v] for v in range(n)] == core.tolist()
    assert rng is not None


def test_planted_clique_survives_kcore(orc):
    rng = np.random.default_rng(2)
    R = random_rotation(rng)
    t = random_translation(rng, 2)
    a_in = rng.uniform(0, 10, (40, 3))
    b_in = a_in @ R.T + t + rng.normal(0, 0.01, (40, 3))
    a_out = rng.uniform(0, 10, (200, 3))
    b_out = rng.uniform(0, 10, (200, 3))
    a = np.concatenate([a_in, a_out])
    b = np.concatenate([b_in, b_out])
    offs, adj = orc.invariant_graph(a, b, beta=0.05)
    keep = orc.max_kcore(offs, adj)
    assert set(range(40)) <= set(keep.tolist())
    Re, te, w = orc.gnc_tls(a[keep], b[keep], 0.05)
    rot, tr = orc.pose_errors(Re, te, R, t)
    assert rot < 0.5 and tr < 0.05


def test_gnc_tls_with_outliers(orc):
    rng = np.random.default_rng(3)
    R = random_rotation(rng)
    t = random_translation(rng, 2)
    a = rng.uniform(-5, 5, (100, 3))
    b = a @ R.T + t + rng.normal(0, 0.01, (100, 3))
    b[:30] = rng.uniform(-5, 5, (30, 3))
    Re, te, w = orc.gnc_tls(a, b, 0.1)
    rot, tr = orc.pose_errors(Re, te, R, t)
    assert rot < 0.5 and tr < 0.05
    assert w[:30].max() < 0.5 and w[30:].min() > 0.5


def test_end_to_end_registers_clutter_scene(orc):
    src, tgt, R, t, vps, vpt = scene_pair(3, n=12000, clutter=True)
    A, fs, ft, vs, vt = orc.front_end(src, tgt, 0.1, vps, vpt)
    Re, te, n_in = orc.register(A, vs, vt, 0.1)
    assert orc.is_success(Re, te, R, t)
    assert n_in >= 10


def _corr(rows):
    A = np.zeros(len(rows), dtype=[("i", np.int32), ("j", np.int32), ("d1", np.float64), ("d2", np.float64)])
    for k, (i, d1, d2) in enumerate(rows):
        A[k] = (i, 100 + i, d1, d2)
    return A


def test_ratio_filter_planted_order(orc):
    """Sec. III-D keeps the N_tau correspondences with the lowest d1/d2
    (Lowe's ratio).  The expected lists below are worked out by hand:
    ratios 8: 0, 3: 0.1, 7: 0.25, 9: 0.25, 5: 0.5, 2: 0.75, 1: 1 (d2 = 0,
    read as 1), 4: 1.  Equal ratios keep the lower i first.  A filter that
    took d2/d1, sorted descending, broke ties to the higher i or sent d2 = 0
    to the end would return another list."""
    A = _corr([(7, 1.0, 4.0), (2, 3.0, 4.0), (5, 1.0, 2.0), (9, 2.0, 8.0), (1, 0.0, 0.0), (4, 2.0, 2.0),
               (3, 1.0, 10.0), (8, 0.0, 5.0)])
    assert orc.ratio_filter(A, 4)["i"].tolist() == [8, 3, 7, 9]
    assert orc.ratio_filter(A, 7)["i"].tolist() == [8, 3, 7, 9, 5, 2, 1]
    assert orc.ratio_filter(A, 8)["i"].tolist() == [8, 3, 7, 9, 5, 2, 1, 4]
    assert orc.ratio_filter(A, 100)["i"].tolist() == [8, 3, 7, 9, 5, 2, 1, 4]
    # the rows travel whole: j and the distances stay with their i
    kept = orc.ratio_filter(A, 2)
    assert kept["j"].tolist() == [108, 103] and kept["d2"].tolist() == [5.0, 10.0]


def test_ratio_filter_more_than_n_tau(orc):
    """More correspondences than the paper's N_tau = 3000 (Sec. IV-B): the
    ratios are a planted permutation p of 0..3499 (ratio p/4000), so the kept
    rows are exactly those with p < 3000, in increasing p."""
    rng = np.random.default_rng(5)
    n = 3500
    p = rng.permutation(n)
    rows = [(int(i), float(p[i]), 4000.0) for i in range(n)]
    A = _corr(rows)
    kept = orc.ratio_filter(A, 3000)
    expect = np.empty(n, np.int64)
    expect[p] = np.arange(n)  # expect[k] = the i whose planted rank is k
    assert kept["i"].tolist() == expect[:3000].tolist()


def test_invariant_graph_edge_at_two_beta(orc):
    """Eq. 3 joins two correspondences when the lengths of their source and
    target segments differ by at most 2 beta.  Lengths are exact binary
    fractions: with beta = 0.25 a difference of 0.5 (= 2 beta) is an edge,
    0.375 (= 1.5 beta, which a test against beta alone would reject) is an
    edge, 0.625 is not."""
    a = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 0, 0], [1.0, 0, 0], [0.0, 0, 0], [1.0, 0, 0]])
    for db, edge in ((1.5, True), (1.375, True), (1.625, False), (0.5, True), (0.375, False)):
        b = np.array([[0.0, 0, 0], [db, 0, 0]])
        offs, adj = orc.invariant_graph(a[:2], b, beta=0.25)
        assert (offs[1] - offs[0] == 1) == edge, (db, edge)
        assert offs[-1] == (2 if edge else 0)
