"""kmx_suppress_ground (geometric suppression, Sec. III-B) against the
oracle's stand-in: every decision of both is exact or a fixed sequence of
IEEE FP64 operations, so the ground flags, the per-bin planes (a, b, c and
status, bit for bit) and the kept cloud must be identical.  Then the chain
suppress -> voxelise (device count) against the oracle, and registration of
LiDAR pairs that fail without suppression."""
import numpy as np
import pytest

from oracle import ground as G
from synth import lidar_pair

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


def _disc(rmax=30.0, step=0.3, z=-1.73, f=None):
    g = np.arange(-rmax, rmax, step)
    xx, yy = np.meshgrid(g, g)
    x, y = xx.ravel(), yy.ravel()
    keep = (x * x + y * y >= 2.8 ** 2) & (x * x + y * y < (rmax - 0.5) ** 2)
    x, y = x[keep], y[keep]
    zz = np.full(x.shape, z) if f is None else f(x, y)
    return np.stack([x, y, zz], 1).astype(np.float32)


def _edges():
    """Points on and next to every ring edge and on the sector edges that are
    exact in both precisions (axes, diagonals): the index decisions the GPU
    takes in FP32 must fall back to the FP64 definition there."""
    zr = (2.7, 12.3, 22.1, 41.1, 80.0)
    rings = (2, 4, 4, 4)
    radii = []
    for k in range(4):
        for j in range(rings[k] + 1):
            r = np.float32(zr[k] + j * (zr[k + 1] - zr[k]) / rings[k])
            radii += [np.nextafter(r, np.float32(0)), r, np.nextafter(r, np.float32(100))]
    ang = np.concatenate([np.arange(8) * np.pi / 4, np.random.default_rng(2).uniform(0, 2 * np.pi, 40)])
    pts = np.array([[r * np.cos(a), r * np.sin(a), -1.73] for r in radii for a in ang], np.float32)
    d = np.float32(7.0)
    exact = np.array([[d, d, -1.73], [-d, d, -1.73], [-d, -d, -1.73], [d, -d, -1.73], [d, 0, -1.73], [0, d, -1.73],
                      [-d, 0, -1.73], [0, -d, -1.73], [-0.0, d, -1.73], [d, -0.0, -1.73]], np.float32)
    return np.concatenate([pts, exact, _disc(step=0.5)])


def _cases():
    rng = np.random.default_rng(5)
    walls = np.concatenate([np.stack([8 + 2 * np.linspace(0, 1, 40), np.full(40, 5.0), np.full(40, zc)], 1)
                            for zc in np.linspace(-1.73, 1.0, 30)]).astype(np.float32)
    slope = np.stack(np.meshgrid(np.arange(4.0, 6.0, 0.05), np.arange(0.2, 0.8, 0.05)), -1).reshape(-1, 2)
    slope = np.concatenate([slope, (0.7 * (slope[:, :1] - 5.0) - 1.7)], 1).astype(np.float32)
    noisy = _disc(step=0.2, f=lambda x, y: 0.02 * x - 1.7 + rng.normal(0, 0.03, x.shape))
    return {
        "flat_walls": np.concatenate([_disc(), walls]),
        "tilted": _disc(f=lambda x, y: 0.015 * x - 0.01 * y - 1.8),
        "steep": _disc(f=lambda x, y: 1.5 * y - 1.7),
        "roof": _disc(z=0.5),
        "slope35": slope,
        "noisy": noisy,
        "lidar_a": lidar_pair(1000)[0],
        "lidar_b": lidar_pair(1003, az_bins=1024)[1],
        "tiny": np.array([[5.0, 0.3, -1.7], [5.1, 0.4, -1.7]], np.float32),
        # points 10 m below the ground: the GPU's lowest-point window (8 m)
        # no longer holds the n_lpr lowest, so it takes its other path
        "deep_outliers": np.concatenate([_disc(), np.array([[5.0, 0.5, -11.73], [10.0, -3.0, -12.5]], np.float32)]),
        "edges": _edges(),
    }


def _check(torch, kmx, ctx, pts, stride=3, prm=None, oprm=None):
    x = np.zeros((len(pts), stride), np.float32)
    x[:, :3] = pts
    if stride == 4:
        x[:, 3] = np.arange(len(pts))
    o = G.suppress_ground(pts, oprm)
    r = ctx.suppress_ground(torch.from_numpy(x).cuda(), prm, want_ground=True, want_planes=True)
    ctx.sync()
    n = len(pts)
    assert int(r["n_out"].item()) == int((~o["ground"]).sum())
    assert np.array_equal(r["ground"][:n].cpu().numpy().astype(bool), o["ground"])
    gp = r["planes"].cpu().numpy()
    assert np.array_equal(gp.view(np.uint64), o["planes"].view(np.uint64)), \
        "plane rows differ: %s" % np.nonzero((gp != o["planes"]).any(1))[0][:5]
    kept = r["out"][: int(r["n_out"].item())].cpu().numpy()
    assert np.array_equal(kept[:, :3].view(np.uint32), o["kept"].view(np.uint32))
    if stride == 4:
        assert np.array_equal(kept[:, 3], np.nonzero(~o["ground"])[0].astype(np.float32))
    return o


@pytest.mark.parametrize("case", ["flat_walls", "tilted", "steep", "roof", "slope35", "noisy", "lidar_a",
                                  "lidar_b", "tiny", "deep_outliers", "edges"])
def test_suppression_bit_exact(env, case):
    torch, kmx, ctx = env
    o = _check(torch, kmx, ctx, _cases()[case])
    if case.startswith("lidar"):
        assert o["ground"].mean() > 0.5 and (o["planes"][:, 3] == 4).sum() > 100


def test_suppression_stride4_params_and_empty(env):
    torch, kmx, ctx = env
    pts = lidar_pair(1001)[0]
    _check(torch, kmx, ctx, pts, stride=4)
    # non-default parameters, mirrored on both sides
    prm = kmx.ground_params_default(th_seeds=0.3, th_dist=0.2, n_iter=1, n_lpr=5, quant_log2=7, max_ground_z=-1.2)
    oprm = G.GroundParams(th_seeds=0.3, th_dist=0.2, n_iter=1, n_lpr=5, quant_log2=7, max_ground_z=-1.2)
    _check(torch, kmx, ctx, pts, prm=prm, oprm=oprm)
    # no points
    r = ctx.suppress_ground(torch.zeros((0, 3), dtype=torch.float32, device="cuda"), want_planes=True)
    ctx.sync()
    assert int(r["n_out"].item()) == 0 and np.all(r["planes"].cpu().numpy() == 0)


def test_suppression_rejects_bad_arguments(env):
    torch, kmx, ctx = env
    x = torch.zeros((10, 3), dtype=torch.float32, device="cuda")
    p = kmx.ground_params_default()
    p.zone_r[1] = 1.0  # not increasing
    assert kmx.ground_bins(p) == -1
    with pytest.raises(kmx.KmxError) as e:
        ctx.suppress_ground(x, p)
    assert e.value.status == kmx.KMX_EINVAL
    p = kmx.ground_params_default(quant_log2=10)  # 80 m * 2^10 overflows the 16-bit coordinate range
    with pytest.raises(kmx.KmxError) as e:
        ctx.suppress_ground(x, p)
    assert e.value.status == kmx.KMX_EINVAL
    with pytest.raises(kmx.KmxError) as e:
        ctx.suppress_ground(x, out=x)  # in place is refused
    assert e.value.status == kmx.KMX_EINVAL
    ctx.sync()


def test_suppress_then_voxelise_on_device_count(env, orc):
    torch, kmx, ctx = env
    from paper_2409_15615_gb300 import pipeline

    src = lidar_pair(1002)[0]
    cs = pipeline.CloudState(ctx, len(src))
    cs.suppress = kmx.ground_params_default()
    cs.raw.copy_(torch.from_numpy(src).cuda())
    prm = kmx.params_default(0.3)
    cs.features(len(src), prm)
    ctx.sync()
    vs, _ = orc.voxelize(G.suppress_ground(src)["kept"], 0.3)
    nv = int(cs.n_vox.item())
    assert nv == len(vs)
    assert np.array_equal(cs.vox4[:nv].cpu().numpy().view(np.uint32), vs.view(np.uint32))
    # the plain voxeliser on the same kept rows gives the same cloud
    out4, n_out, _ = ctx.voxelize(cs.kept[: int(cs.n_kept.item())], 0.3)
    ctx.sync()
    assert np.array_equal(out4[:nv].cpu().numpy().view(np.uint32), vs.view(np.uint32))


@pytest.mark.parametrize("seed", [1000, 1001, 1002])
def test_lidar_pair_registers_after_suppression(env, seed):
    """Features, matching, pruning and GNC on the device: LiDAR pairs whose
    ground dominates the maximum k-core register once it is removed, as the
    oracle's chain does on the same suppressed clouds."""
    torch, kmx, ctx = env
    from oracle import registration as reg
    from paper_2409_15615_gb300 import pipeline

    src, tgt, R, t, vps, vpt = lidar_pair(seed)
    pair = pipeline.PairState(ctx, len(src), len(tgt))
    pair.src.suppress = pair.tgt.suppress = kmx.ground_params_default()
    pair.src.raw.copy_(torch.from_numpy(src).cuda())
    pair.tgt.raw.copy_(torch.from_numpy(tgt).cuda())
    ps = kmx.params_default(0.3, viewpoint=np.float32(vps).tolist())
    pt = kmx.params_default(0.3, viewpoint=np.float32(vpt).tolist())
    pair.run_checked(len(src), len(tgt), ps, pt, kmx.MATCH_FP32_EXACT)
    pr = ctx.prune(pair.corr, int(pair.n_corr.item()), pair.src.vox4, pair.tgt.vox4, 0.45)
    g = ctx.gnc(pair.corr, pr, pair.src.vox4, pair.tgt.vox4, 0.45)
    ctx.sync()
    Rg = g["R"].cpu().numpy().reshape(3, 3)
    tg = g["t"].cpu().numpy()
    pair.close()
    assert g["stats"].cpu().numpy()[3] == 0
    assert reg.is_success(Rg, tg, R, t)
    rot, tr = reg.pose_errors(Rg, tg, R, t)
    assert rot < 1.0 and tr < 0.3
