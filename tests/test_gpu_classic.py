"""Classic FPFH baseline (Sec. III-C, Fig. 2(a)) through the C ABI against the
oracle's classic FPFH on the same voxelised clouds.

The GPU stage computes its own normals (three searches, nothing passed in), so
the descriptors are compared chained: J and the PCA flags exactly, normals
within 1e-5 rad outside the ill-posed bands, and every SPFH / FPFH row within
1e-4 at the 100-per-histogram scale plus the exact allowance of the pairs
whose bins a normal error of up to 1e-5 rad (or an ill-posed normal) can move.
"""
import numpy as np
import pytest

from parity_helpers import chained_pair_prone, fpfh_allowance, hist_violation, spfh_allowance
from synth import lidar_pair, scene_pair

pytestmark = pytest.mark.gpu

H = 11
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


def _bands(c, pts, vp):
    ev, n4 = c["evals"], c["normal4"]
    l1, l2, l3 = ev[:, 0], ev[:, 1], ev[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        degenerate = (l2 - l3) / np.where(l1 > 0, l1, 1) < 1e-2
        view = vp[None, :] - pts[:, :3].astype(np.float64)
        sign_ill = np.abs(np.sum(n4[:, :3] * view, 1)) / np.maximum(np.linalg.norm(view, axis=1), 1e-300) < 1e-4
    return degenerate | sign_ill


@pytest.mark.parametrize("case", ["scene", "lidar", "plane_pole"])
def test_classic_fpfh_parity(env, orc, case):
    torch, kmx, ctx = env
    if case == "scene":
        src, _, _, _, vp, _ = scene_pair(6)
        v = 0.1
    elif case == "lidar":
        src, _, _, _, vp, _ = lidar_pair(6)
        v = 0.3
    else:
        g = np.arange(40) * 0.1
        xx, yy = np.meshgrid(g, g)
        plane = np.stack([xx.ravel(), yy.ravel(), 0.01 * np.sin(xx.ravel() * 3)], 1)
        pole = np.stack([np.full(30, 9.0), np.full(30, 9.0), np.arange(30) * 0.1], 1)
        src, vp, v = np.concatenate([plane, pole]).astype(np.float32), np.array([2.0, 2.0, 6.0]), 0.1
    vs, _ = orc.voxelize(src, v)
    vp32 = np.asarray(vp, np.float32)
    prm = kmx.params_default(v, viewpoint=vp32.tolist())
    oprm = orc.OracleParams(v, viewpoint=vp32.astype(np.float64))
    c = orc.classic_fpfh(vs, oprm)
    p = torch.from_numpy(vs).cuda()
    grid = ctx.build_grid(p, prm.r_fpfh)
    res = ctx.fpfh_classic(grid, prm, want_spfh=True)
    ctx.sync()
    n = len(vs)
    nJ = int(res["n_valid"].item())
    gJ = res["valid"][:nJ].cpu().numpy()
    g_fl = res["flags"][:n].cpu().numpy()
    # the point set and the PCA flag depend on integer counts only
    assert np.array_equal(gJ, c["J"])
    assert np.array_equal(g_fl & 4, c["flags"] & 4)
    assert np.array_equal((g_fl & 1) > 0, (c["flags"] & 1) > 0)
    assert np.array_equal((g_fl & 2) > 0, (g_fl & 1) > 0)
    # normals
    has = (c["flags"] & 1) > 0
    ill = _bands(c, vs, oprm.viewpoint) & has
    g_n4 = res["normal4"][:n].cpu().numpy()
    chk = has & ~ill
    a = g_n4[chk, :3].astype(np.float64)
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = c["normal4"][chk, :3]
    ang = np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.sum(a * b, 1))
    assert ang.max() <= NORMAL_TOL_RAD, "max normal angle %.3g rad" % ang.max()
    assert np.all(g_n4[~has] == 0)
    # descriptors, every row, with the chained allowance
    n_marg = chained_pair_prone(vs, c["normal4"], has, ill, c["voffs"], c["vnbr"], NORMAL_TOL_RAD)
    a_sp = spfh_allowance(n_marg, c["npairs"])
    gsp = res["spfh"][:n, :33].cpu().numpy().astype(np.float64)
    v_sp = hist_violation(gsp, c["spfh"], a_sp)
    assert v_sp.max() <= 1.0, "SPFH off by %.3g x tolerance" % v_sp.max()
    assert np.all(res["spfh"][:n, 33:].cpu().numpy() == 0)
    a_fp = fpfh_allowance(vs, c["J"], c["voffs"], c["vnbr"], a_sp)
    gfp = res["desc"][:nJ, :33].cpu().numpy().astype(np.float64)
    v_fp = hist_violation(gfp, c["fpfh"], a_fp)
    assert v_fp.max() <= 1.0, "FPFH off by %.3g x tolerance" % v_fp.max()
    assert np.all(res["desc"][:nJ, 33:].cpu().numpy() == 0)
    clean = a_sp[has] == 0
    assert clean.mean() > {"scene": 0.6, "lidar": 0.2, "plane_pole": 0.3}[case]
    assert hist_violation(gsp[has][clean], c["spfh"][has][clean]).max() <= 1.0


def test_classic_keeps_what_fasterpfh_drops(env, orc):
    """On a LiDAR scan the classic baseline describes every point with a
    normal, Faster-PFH only the reliable ones (Sec. III-C's second change)."""
    torch, kmx, ctx = env
    src, _, _, _, vp, _ = lidar_pair(3)
    vs, _ = orc.voxelize(src, 0.3)
    prm = kmx.params_default(0.3, viewpoint=np.float32(vp).tolist())
    p = torch.from_numpy(vs).cuda()
    grid = ctx.build_grid(p, prm.r_fpfh)
    cl = ctx.fpfh_classic(grid, prm)
    nb = ctx.normals(grid, prm, len(vs) * 200)
    fp = ctx.fasterpfh(grid, prm, nb["normal4"], nb["flags"], nb["offs"], nb["nbr"])
    ctx.sync()
    jc = cl["valid"][: int(cl["n_valid"].item())].cpu().numpy()
    jf = fp["valid"][: int(fp["n_valid"].item())].cpu().numpy()
    assert np.all(np.isin(jf, jc)) and len(jc) > len(jf)


def test_classic_empty_and_bad_grid(env):
    torch, kmx, ctx = env
    prm = kmx.params_default(0.1)
    p = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    n0 = torch.zeros(1, dtype=torch.int64, device="cuda")
    grid = ctx.build_grid(p, prm.r_fpfh, n_cap=4, d_n=n0)
    res = ctx.fpfh_classic(grid, prm)
    ctx.sync()
    assert int(res["n_valid"].item()) == 0
    small = ctx.build_grid(p, prm.r_fpfh * 0.5)
    with pytest.raises(kmx.KmxError) as e:
        ctx.fpfh_classic(small, prm)
    assert e.value.status == kmx.KMX_EINVAL
    ctx.sync()
