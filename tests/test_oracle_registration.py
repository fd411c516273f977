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
