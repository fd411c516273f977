"""The bench's per-result FP64 check (`bench.precision_vs_fp64`) on a CPU
stand-in of a pair: correspondences built from the exact FP64 nearest rows
must report full agreement and FP32-level relative errors; a planted wrong
partner must lower the agreement, and squared distances in place of the
Euclidean ones kmx_corr holds must show as large relative errors."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _fake_pair(P, Q, JP, JQ, gi, gj, d1, d2):
    def side(desc, J):
        d = np.zeros((len(desc), 36), np.float32)
        d[:, :33] = desc
        return types.SimpleNamespace(out=dict(desc=torch.from_numpy(d), valid=torch.from_numpy(J.astype(np.int32)),
                                              n_valid=torch.tensor([len(J)], dtype=torch.int64)))

    pair = types.SimpleNamespace(src=side(P, JP), tgt=side(Q, JQ))
    pair.correspondences = lambda: (gi, gj, d1, d2)
    return pair


def _case(seed=3, n=300, m=400):
    rng = np.random.default_rng(seed)
    P = rng.gamma(0.5, 20.0, (n, 33)).astype(np.float32)
    Q = rng.gamma(0.5, 20.0, (m, 33)).astype(np.float32)
    JP = np.sort(rng.choice(5 * n, n, replace=False))
    JQ = np.sort(rng.choice(5 * m, m, replace=False))
    D = ((P.astype(np.float64)[:, None, :] - Q.astype(np.float64)[None, :, :]) ** 2).sum(2)
    nn = D.argmin(1)
    srt = np.sort(D, axis=1)
    gi, gj = JP, JQ[nn]
    d1 = np.sqrt(srt[:, 0]).astype(np.float32)  # kmx_corr holds Euclidean distances
    d2 = np.sqrt(srt[:, 1]).astype(np.float32)
    return P, Q, JP, JQ, gi, gj, d1, d2, nn


def test_exact_partners_agree():
    import bench

    P, Q, JP, JQ, gi, gj, d1, d2, _ = _case()
    r = bench.precision_vs_fp64(_fake_pair(P, Q, JP, JQ, gi, gj, d1, d2), rows=120)
    assert r["rows"] == 120 and r["nn_equal_fp64"] == 1.0
    assert r["d1_rel_err_max"] < 1e-6 and r["d2_rel_err_max"] < 1e-6


def test_planted_wrong_partner_is_seen():
    import bench

    P, Q, JP, JQ, gi, gj, d1, d2, nn = _case()
    gj = gj.copy()
    gj[::2] = JQ[(nn[::2] + 1) % len(JQ)]  # half the partners moved to another row
    r = bench.precision_vs_fp64(_fake_pair(P, Q, JP, JQ, gi, gj, d1, d2), rows=300)
    assert r["nn_equal_fp64"] < 0.6
    assert r["d1_rel_err_max"] > 1e-3  # the stated d1 no longer matches the returned pair


def test_squared_distances_are_seen():
    import bench

    P, Q, JP, JQ, gi, gj, d1, d2, _ = _case()
    r = bench.precision_vs_fp64(_fake_pair(P, Q, JP, JQ, gi, gj, d1 * d1, d2 * d2), rows=120)
    assert r["nn_equal_fp64"] == 1.0
    assert r["d1_rel_err_median"] > 1.0 and r["d2_rel_err_median"] > 1.0
