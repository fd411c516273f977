"""kmx_gnc (Sec. III-E, GNC-TLS around Horn's closed form) against the
oracle's FP64 GNC-TLS (SVD alignment) on the same maximum k-core.  The GPU
works in FP32 on centred coordinates, so the poses are compared within
tolerance; the success verdict of Sec. IV-A must be the same."""
import math

import numpy as np
import pytest

from synth import lidar_pair, scene_pair

pytestmark = pytest.mark.gpu

ROT_TOL = 1e-4  # rad
TRANS_TOL = 1e-3  # m


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


def _angle(Ra, Rb):
    """Rotation angle between Ra and Rb; for small angles from the Frobenius
    norm of Ra^T Rb - I (= sqrt(2) * 2 sin(angle / 2)), which acos of the
    trace cannot resolve below ~1e-4 rad."""
    D = np.asarray(Ra).T @ np.asarray(Rb)
    s = np.linalg.norm(D - np.eye(3)) / (2.0 * math.sqrt(2.0))
    return 2.0 * math.asin(min(1.0, s))


def _device_problem(torch, a, b):
    """corr / selection / inlier arrays that make point k = (a[k], b[k])."""
    n = len(a)
    c = np.zeros((max(n, 1), 4), np.int32)
    c[:n, 0] = np.arange(n)
    c[:n, 1] = np.arange(n)
    s4 = np.zeros((max(n, 1), 4), np.float32)
    t4 = np.zeros((max(n, 1), 4), np.float32)
    s4[:n, :3], t4[:n, :3] = a, b
    idx = torch.arange(max(n, 1), dtype=torch.int32, device="cuda")
    pruned = dict(sel=idx, inlier=idx.clone(), n_inlier=torch.tensor([n], dtype=torch.int64, device="cuda"))
    return torch.from_numpy(c).cuda(), pruned, torch.from_numpy(s4).cuda(), torch.from_numpy(t4).cuda()


def _compare(got, R, t, w):
    Rg = got["R"].cpu().numpy().reshape(3, 3)
    tg = got["t"].cpu().numpy()
    assert _angle(Rg, R) < ROT_TOL
    assert np.linalg.norm(tg - t) < TRANS_TOL
    n = len(w)
    wg = got["w"][:n].cpu().numpy()
    disagree = np.count_nonzero((wg > 0.5) != (np.asarray(w) > 0.5))
    assert disagree <= max(2, n // 100)


@pytest.mark.parametrize("case", ["lidar", "scene"])
def test_gnc_on_pipeline_pairs(env, case):
    torch, kmx, ctx = env
    from oracle import registration as reg
    from paper_2409_15615_gb300 import pipeline

    if case == "lidar":
        (src, tgt, Rgt, tgt_t, vps, vpt), v = lidar_pair(8), 0.3
    else:
        (src, tgt, Rgt, tgt_t, vps, vpt), v = scene_pair(500, n=10000, clutter=True), 0.1
    pair = pipeline.PairState(ctx, len(src), len(tgt))
    pair.src.raw.copy_(torch.from_numpy(src).cuda())
    pair.tgt.raw.copy_(torch.from_numpy(tgt).cuda())
    ps = kmx.params_default(v, viewpoint=np.float32(vps).tolist())
    pt = kmx.params_default(v, viewpoint=np.float32(vpt).tolist())
    pair.run_checked(len(src), len(tgt), ps, pt, kmx.MATCH_FP32_EXACT)
    beta = 1.5 * v
    n_corr = int(pair.n_corr.item())
    pr = ctx.prune(pair.corr, n_corr, pair.src.vox4, pair.tgt.vox4, beta)
    got = ctx.gnc(pair.corr, pr, pair.src.vox4, pair.tgt.vox4, beta)
    ctx.sync()
    # the oracle's GNC-TLS on the same maximum k-core
    n_in = int(pr["n_inlier"].item())
    sel = pr["sel"].cpu().numpy()
    inl = pr["inlier"][:n_in].cpu().numpy()
    corr = pair.corr[:n_corr].cpu().numpy()
    rows = corr[sel[inl]]
    vs = pair.src.vox4[: int(pair.src.n_vox.item())].cpu().numpy().astype(np.float64)
    vt = pair.tgt.vox4[: int(pair.tgt.n_vox.item())].cpu().numpy().astype(np.float64)
    a, b = vs[rows[:, 0], :3], vt[rows[:, 1], :3]
    R, t, w = reg.gnc_tls(a, b, beta)
    _compare(got, R, t, w)
    st = got["stats"].cpu().numpy()
    assert st[2] == n_in and st[3] == 0
    Rg = got["R"].cpu().numpy().reshape(3, 3)
    assert reg.is_success(Rg, got["t"].cpu().numpy(), Rgt, tgt_t) == reg.is_success(R, t, Rgt, tgt_t)
    pair.close()


@pytest.mark.parametrize("n,outlier_frac", [(1829, 0.3), (500, 0.0), (4096, 0.5), (40, 0.2)])
def test_gnc_planted(env, n, outlier_frac):
    torch, kmx, ctx = env
    from oracle import registration as reg

    rng = np.random.default_rng(n)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w0, x, y, z = q
    Rt = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w0), 2 * (x * z + y * w0)],
                   [2 * (x * y + z * w0), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w0)],
                   [2 * (x * z - y * w0), 2 * (y * z + x * w0), 1 - 2 * (x * x + y * y)]])
    tt = rng.uniform(-20, 20, 3)
    a = rng.uniform(-40, 40, (n, 3))
    b = a @ Rt.T + tt + rng.normal(0, 0.05, (n, 3))
    k = int(n * outlier_frac)
    b[:k] = rng.uniform(-60, 60, (k, 3))
    a, b = a.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
    dc, pr, ds, dt = _device_problem(torch, a, b)
    got = ctx.gnc(dc, pr, ds, dt, 0.45, inlier_cap=n)
    ctx.sync()
    R, t, w = reg.gnc_tls(a, b, 0.45)
    _compare(got, R, t, w)
    assert _angle(got["R"].cpu().numpy().reshape(3, 3), Rt) < 1e-2


def test_gnc_too_few_points(env):
    torch, kmx, ctx = env
    a = np.zeros((2, 3))
    dc, pr, ds, dt = _device_problem(torch, a, a)
    got = ctx.gnc(dc, pr, ds, dt, 0.45, inlier_cap=2)
    ctx.sync()
    assert np.array_equal(got["R"].cpu().numpy(), np.eye(3).ravel())
    assert got["stats"].cpu().numpy()[3] == 1


def test_device_registration_success_parity(env):
    """Features, matching, pruning and GNC all on the device: the success
    verdict of Sec. IV-A equals the oracle's whole chain, pair by pair."""
    torch, kmx, ctx = env
    from oracle import core as orc
    from oracle import registration as reg
    from paper_2409_15615_gb300 import pipeline

    flags_o, flags_g = [], []
    for seed in range(500, 512):
        src, tgt, Rgt, tgt_t, vps, vpt = scene_pair(seed, n=10000, clutter=True)
        v = 0.1
        A, fs, ft, vs, vt = orc.front_end(src, tgt, v, np.float32(vps).astype(np.float64),
                                          np.float32(vpt).astype(np.float64))
        Ro, to, _ = reg.register(A, vs, vt, v)
        flags_o.append(reg.is_success(Ro, to, Rgt, tgt_t))
        pair = pipeline.PairState(ctx, len(src), len(tgt))
        pair.src.raw.copy_(torch.from_numpy(src).cuda())
        pair.tgt.raw.copy_(torch.from_numpy(tgt).cuda())
        ps = kmx.params_default(v, viewpoint=np.float32(vps).tolist())
        pt = kmx.params_default(v, viewpoint=np.float32(vpt).tolist())
        pair.run_checked(len(src), len(tgt), ps, pt, kmx.MATCH_FP32_EXACT)
        pr = ctx.prune(pair.corr, int(pair.n_corr.item()), pair.src.vox4, pair.tgt.vox4, 1.5 * v)
        got = ctx.gnc(pair.corr, pr, pair.src.vox4, pair.tgt.vox4, 1.5 * v)
        ctx.sync()
        Rg = got["R"].cpu().numpy().reshape(3, 3)
        ok = got["stats"].cpu().numpy()[3] == 0 and reg.is_success(Rg, got["t"].cpu().numpy(), Rgt, tgt_t)
        flags_g.append(bool(ok))
        pair.close()
    assert flags_g == flags_o
    assert sum(flags_o) >= len(flags_o) // 2
