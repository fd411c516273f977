"""kmx_features (Algorithm 1 and Eqs. A2-A5 without stored neighbour lists,
the default hot path) against the list-based kmx_normals + kmx_fasterpfh,
which visits the same neighbours in the same order: every output must be
bit-identical.  And against the oracle's Faster-PFH, chained: J up to the
tau_lin band, normals within 1e-5 rad outside the ill-posed bands, every FPFH
row within 1e-4 at the 100-per-histogram scale plus the allowance of the
pairs a normal error of up to 1e-5 rad can move."""
import numpy as np
import pytest

from parity_helpers import chained_pair_prone, fpfh_allowance, hist_violation, spfh_allowance
from synth import indoor_pair, lidar_pair, scene_pair

pytestmark = pytest.mark.gpu

NORMAL_TOL_RAD = 1e-5


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


def _cloud(orc, case):
    if case == "scene":
        src, _, _, _, vp, _ = scene_pair(7)
        v = 0.1
    elif case == "lidar":
        src, _, _, _, vp, _ = lidar_pair(7)
        v = 0.3
    elif case == "indoor":
        src, _, _, _, vp, _ = indoor_pair(3, n=300000)
        v = 0.02
    else:
        # lattice with spacing 1/8 and r_FPFH = 0.5: many distances on the radius
        g = np.arange(-6, 7) * 0.125
        xx, yy, zz = np.meshgrid(g, g, g[:5])
        src = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(np.float32)
        vp, v = np.array([0.3, 0.2, 5.0]), 0.1
    vs, _ = orc.voxelize(src, v)
    return vs, np.asarray(vp, np.float32), v


@pytest.mark.parametrize("case", ["scene", "lidar", "indoor", "lattice"])
def test_features_equal_list_path(env, orc, case):
    torch, kmx, ctx = env
    vs, vp, v = _cloud(orc, case)
    prm = kmx.params_default(v, viewpoint=vp.tolist())
    if case == "lattice":
        prm.r_fpfh, prm.r_normal = 0.5, 0.375
    p = torch.from_numpy(vs).cuda()
    grid = ctx.build_grid(p, prm.r_fpfh)
    a = ctx.features(grid, prm, want_spfh=True)
    nb = ctx.normals(grid, prm, len(vs) * 400)
    b = ctx.fasterpfh(grid, prm, nb["normal4"], nb["flags"], nb["offs"], nb["nbr"], want_spfh=True)
    ctx.sync()
    n = len(vs)
    nJ = int(a["n_valid"].item())
    assert nJ == int(b["n_valid"].item()) and nJ > 0
    same = lambda x, y: np.array_equal(x.cpu().numpy().view(np.uint8), y.cpu().numpy().view(np.uint8))
    assert same(a["normal4"][:n], nb["normal4"][:n])
    assert same(a["flags"][:n], nb["flags"][:n])
    assert same(a["valid"][:nJ], b["valid"][:nJ])
    assert same(a["spfh"][:n], b["spfh"][:n])
    assert same(a["desc"][:nJ], b["desc"][:nJ])


@pytest.mark.parametrize("case", ["scene", "lidar"])
def test_features_vs_oracle(env, orc, case):
    torch, kmx, ctx = env
    vs, vp, v = _cloud(orc, case)
    prm = kmx.params_default(v, viewpoint=vp.tolist())
    oprm = orc.OracleParams(v, viewpoint=vp.astype(np.float64))
    f = orc.faster_pfh(vs, oprm)
    p = torch.from_numpy(vs).cuda()
    grid = ctx.build_grid(p, prm.r_fpfh)
    g = ctx.features(grid, prm)
    ctx.sync()
    n = len(vs)
    g_fl = g["flags"][:n].cpu().numpy()
    assert np.array_equal(g_fl & 4, f["flags"] & 4)
    # ill-posed normals and the tau_lin band
    ev, n4 = f["evals"], f["normal4"]
    with np.errstate(divide="ignore", invalid="ignore"):
        ill = (ev[:, 1] - ev[:, 2]) / np.where(ev[:, 0] > 0, ev[:, 0], 1) < 1e-2
        view = oprm.viewpoint[None, :] - vs[:, :3].astype(np.float64)
        ill |= np.abs(np.sum(n4[:, :3] * view, 1)) / np.maximum(np.linalg.norm(view, axis=1), 1e-300) < 1e-4
    lin_band = np.abs(n4[:, 3] - oprm.tau_lin) < 1e-5
    pca = (f["flags"] & 4) > 0
    chk = pca & ~ill & (ev[:, 0] > 0)
    a = g["normal4"][:n].cpu().numpy()[chk, :3].astype(np.float64)
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    ang = np.arctan2(np.linalg.norm(np.cross(a, n4[chk, :3]), axis=1), np.sum(a * n4[chk, :3], 1))
    assert ang.max() <= NORMAL_TOL_RAD
    B_o, B_g = (f["flags"] & 1) > 0, (g_fl & 1) > 0
    assert np.all((B_o == B_g) | lin_band | ill)
    nJ = int(g["n_valid"].item())
    gJ = g["valid"][:nJ].cpu().numpy()
    diff = np.setxor1d(gJ, f["J"])
    assert len(diff) <= max(2, len(f["J"]) // 1000)
    # rows of J in both whose neighbourhood has the same B on both sides
    bad_b = np.nonzero(B_o != B_g)[0]
    nbr_bad = np.zeros(n, bool)
    if len(bad_b):
        cnt = np.diff(f["offs"])
        owner = np.repeat(np.arange(n), cnt)
        nbr_bad[np.unique(owner[np.isin(f["nbr"], bad_b)])] = True
    row_g = {q: r for r, q in enumerate(gJ)}
    rows = [r for r, q in enumerate(f["J"]) if q in row_g and not nbr_bad[q]]
    assert len(rows) > 0.95 * len(f["J"])
    n_marg = chained_pair_prone(vs, n4, B_o, ill & B_o, f["voffs"], f["vnbr"], NORMAL_TOL_RAD)
    a_fp = fpfh_allowance(vs, f["J"], f["voffs"], f["vnbr"], spfh_allowance(n_marg, f["npairs"]))
    got = g["desc"][torch.as_tensor([row_g[int(f["J"][r])] for r in rows], device="cuda"), :33].cpu().numpy()
    viol = hist_violation(got.astype(np.float64), f["fpfh"][rows], a_fp[rows])
    assert viol.max() <= 1.0, "FPFH off by %.3g x tolerance" % viol.max()
