"""kmx_prune (Sec. III-D) against the oracle's ratio filter, invariant graph
(Eq. 3) and Batagelj-Zaversnik core numbers, on the same correspondence sets:
the selection order, every core number, the largest core number and the
maximum k-core are compared exactly (the k-core decomposition is unique)."""
import numpy as np
import pytest

from synth import lidar_pair, scene_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_15615_gb300 import build, kmx

    build.build()
    ctx = kmx.Context(0)
    yield torch, kmx, ctx
    ctx.close()


def _corr_array(i, j, d1, d2):
    A = np.zeros(len(i), dtype=[("i", np.int64), ("j", np.int64), ("d1", np.float64), ("d2", np.float64)])
    A["i"], A["j"] = i, j
    A["d1"], A["d2"] = np.float32(d1), np.float32(d2)
    return A


def _run_both(torch, ctx, corr_rows, src4, tgt4, beta, n_tau):
    """corr_rows: (i, j, d1, d2) arrays; src4/tgt4: float32 [n][4]."""
    from oracle import registration as reg

    i, j, d1, d2 = (np.asarray(x) for x in corr_rows)
    n = len(i)
    c = np.zeros((max(n, 1), 4), np.int32)
    c[:n, 0], c[:n, 1] = i, j
    c[:n, 2] = np.asarray(d1, np.float32).view(np.int32)
    c[:n, 3] = np.asarray(d2, np.float32).view(np.int32)
    dc = torch.from_numpy(c).cuda()
    ds, dt = torch.from_numpy(np.ascontiguousarray(src4, np.float32)).cuda(), torch.from_numpy(
        np.ascontiguousarray(tgt4, np.float32)).cuda()
    r = ctx.prune(dc, n, ds, dt, beta, n_tau=n_tau)
    ctx.sync()
    n_sel = int(r["n_sel"].item())
    g_sel = r["sel"][:n_sel].cpu().numpy()
    g_core = r["core"][:n_sel].cpu().numpy()
    g_kmax = int(r["kmax"].item())
    g_in = r["inlier"][: int(r["n_inlier"].item())].cpu().numpy()
    # oracle on the same rows
    A = _corr_array(i, j, d1, d2)
    sel = reg.ratio_filter(A, n_tau)
    assert n_sel == len(sel)
    assert np.array_equal(np.stack([i[g_sel], j[g_sel]], 1), np.stack([sel["i"], sel["j"]], 1))
    a = np.asarray(src4, np.float64)[np.asarray(sel["i"], np.int64), :3]
    b = np.asarray(tgt4, np.float64)[np.asarray(sel["j"], np.int64), :3]
    offs, adj = reg.invariant_graph(a, b, beta)
    core = reg.core_numbers(offs, adj)
    assert np.array_equal(g_core, core)
    assert g_kmax == (int(core.max()) if len(core) else 0)
    assert np.array_equal(g_in, reg.max_kcore(offs, adj))
    return dict(n_sel=n_sel, kmax=g_kmax, n_inlier=len(g_in), edges=len(adj) // 2)


def _pipeline_corr(torch, kmx, ctx, src, tgt, v, vps, vpt):
    from paper_2409_15615_gb300 import pipeline

    pair = pipeline.PairState(ctx, len(src), len(tgt))
    pair.src.raw.copy_(torch.from_numpy(src).cuda())
    pair.tgt.raw.copy_(torch.from_numpy(tgt).cuda())
    ps = kmx.params_default(v, viewpoint=np.float32(vps).tolist())
    pt = kmx.params_default(v, viewpoint=np.float32(vpt).tolist())
    pair.run_checked(len(src), len(tgt), ps, pt, kmx.MATCH_FP32_EXACT)
    rows = pair.correspondences()
    vs = pair.src.vox4[: int(pair.src.n_vox.item())].cpu().numpy()
    vt = pair.tgt.vox4[: int(pair.tgt.n_vox.item())].cpu().numpy()
    pair.close()
    return rows, vs, vt


@pytest.mark.parametrize("case", ["lidar", "scene"])
def test_prune_on_pipeline_correspondences(env, case):
    torch, kmx, ctx = env
    if case == "lidar":
        (src, tgt, R, t, vps, vpt), v = lidar_pair(8), 0.3
    else:
        (src, tgt, R, t, vps, vpt), v = scene_pair(500, n=10000, clutter=True), 0.1
    rows, vs, vt = _pipeline_corr(torch, kmx, ctx, src, tgt, v, vps, vpt)
    out = _run_both(torch, ctx, rows, vs, vt, 1.5 * v, 3000)
    assert out["kmax"] > 10 and out["n_inlier"] >= 3


def _planted(rng, n, n_in, noise, spread=20.0):
    a = rng.uniform(-spread, spread, (n, 3))
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                  [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                  [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    b = a @ R.T + rng.uniform(-5, 5, 3)
    b[:n_in] += rng.normal(0, noise, (n_in, 3))
    b[n_in:] = rng.uniform(-spread, spread, (n - n_in, 3))
    src4 = np.zeros((n, 4), np.float32)
    tgt4 = np.zeros((n, 4), np.float32)
    src4[:, :3], tgt4[:, :3] = a, b
    return src4, tgt4


@pytest.mark.parametrize("n,n_in,n_tau", [(5000, 400, 3000), (800, 120, 3000), (2000, 300, 50), (0, 0, 3000),
                                          (1, 1, 3000), (3, 3, 2)])
def test_prune_planted(env, n, n_in, n_tau):
    torch, kmx, ctx = env
    rng = np.random.default_rng(n + n_tau)
    src4, tgt4 = _planted(rng, max(n, 1), n_in, 0.05)
    i = rng.permutation(n).astype(np.int64)
    j = i.copy()
    d2 = rng.uniform(1.0, 50.0, n)
    d1 = d2 * rng.uniform(0.0, 1.0, n)
    d1[:10] = d2[:10] * 0.5  # equal ratios: ties go to the lower i
    if n > 20:
        d2[15:20] = 0.0  # ratio 1 by definition
        d1[15:20] = 0.0
    _run_both(torch, ctx, (i, j, d1, d2), src4, tgt4, 0.45, n_tau)


def test_prune_all_ratios_equal(env):
    """Every ratio in one bucket: the threshold bucket holds every candidate."""
    torch, kmx, ctx = env
    rng = np.random.default_rng(7)
    n = 4000
    src4, tgt4 = _planted(rng, n, 600, 0.02)
    i = np.arange(n, dtype=np.int64)[::-1].copy()
    d = np.full(n, 3.0)
    out = _run_both(torch, ctx, (i, i.copy(), d, d), src4, tgt4, 0.3, 3000)
    assert out["n_sel"] == 3000
