"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: voxel assignments, centroids and neighbour sets bit-exact; normals
within 1e-5 rad; SPFH/FPFH bins within 1e-4 at the 100-per-histogram scale
(1e-4 * S_l / 100 for a sub-histogram whose oracle sum is S_l);
correspondences identical.  Excused are only the cases the oracle marks as
ill-posed at FP32 precision: near-degenerate or sign-ill-posed normals, p_lin
within 1e-5 of tau_lin, matches whose top-2 distance gap is below 1e-3
(relative).  Histogram rows are all checked; a row that contains pairs within
2e-6 (feature units) of a bin edge, the atan2 cut, the source tie or the
degenerate-pair threshold gets the exact extra allowance such a flip causes.
"""
import numpy as np
import pytest

from synth import lidar_pair, scene_pair

pytestmark = pytest.mark.gpu

H = 11
NORMAL_TOL_RAD = 1e-5
BIN_TOL = 1e-4          # at the 100-per-histogram scale
FEATURE_BAND = 2e-6     # f units (FP32 feature error is ~1e-7)
GAP_BAND = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    from paper_2409_15615_gb300 import build, kmx

    build.build()
    c = kmx.Context(0)
    yield c
    c.close()


def dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def params_for(kmx, orc, v, vp):
    vp32 = np.asarray(vp, np.float32)
    return (kmx.params_default(v, viewpoint=vp32.tolist()),
            orc.OracleParams(v, viewpoint=vp32.astype(np.float64)))


# ----------------------------------------------------------------------------
# voxelisation
# ----------------------------------------------------------------------------


def _exponent_mix():
    """Voxels of ~60 members (integer path near its shift limit), voxels
    mixing magnitudes from 1e-30 to 0.5 and subnormals, zeros and -0.0 (FP64
    input-order path), on both sides of the origin."""
    rng = np.random.default_rng(4)
    a = rng.random((4000, 3)) * 2.0
    b = rng.random((300, 3)) * 0.5 * 10.0 ** rng.uniform(-30, 0, (300, 3))
    c = rng.random((40, 3)) * 0.25
    c[:10, 0] = 1e-40  # subnormal in FP32
    c[10:20, 1] = 0.0
    c[20:30, 2] = -0.0
    x = np.concatenate([a, b, c, -a[:500], -b[:100]]).astype(np.float32)
    return x[rng.permutation(len(x))]


@pytest.mark.parametrize("case", ["scene", "lidar", "stride4", "negative", "single", "exponents"])
def test_voxelize_bit_exact(torch_cuda, ctx, orc, case):
    torch = torch_cuda
    if case == "scene":
        x, v = scene_pair(0)[0], 0.1
    elif case == "lidar":
        x, v = lidar_pair(0)[0], 0.3
    elif case == "stride4":
        x = scene_pair(1, n=7000)[1]
        x = np.concatenate([x, np.ones((len(x), 1), np.float32)], 1)
        v = 0.07
    elif case == "negative":
        rng = np.random.default_rng(3)
        x = rng.normal(0, 0.3, (5000, 3)).astype(np.float32)
        x[:50] = (rng.integers(-8, 8, (50, 3)) * 0.125).astype(np.float32)  # exactly on faces
        v = 0.125
    elif case == "exponents":
        x, v = _exponent_mix(), 0.5
    else:
        x, v = np.array([[-1.5, 2.25, 0.0]], np.float32), 0.5
    ref, ref_assign = orc.voxelize(x, v)
    out4, n_out, assign = ctx.voxelize(dev(torch, x), v, assign=True)
    ctx.sync()
    n = int(n_out.item())
    assert n == len(ref)
    got = out4[:n].cpu().numpy()
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert np.array_equal(assign.cpu().numpy()[: len(x)], ref_assign)


def test_voxelize_empty_and_range(torch_cuda, ctx):
    torch = torch_cuda
    from paper_2409_15615_gb300 import kmx

    out4, n_out, _ = ctx.voxelize(torch.zeros((0, 3), device="cuda"), 0.1, cap=4)
    ctx.sync()
    assert int(n_out.item()) == 0
    big = np.array([[0, 0, 0], [2.0 ** 20 * 0.1 + 10.0, 0, 0]], np.float32)
    ctx.voxelize(dev(torch, big), 0.1)
    with pytest.raises(kmx.KmxError) as e:
        ctx.sync()
    assert e.value.status == kmx.KMX_ERANGE


# ----------------------------------------------------------------------------
# radius search and normals (Algorithm 1, step 1)
# ----------------------------------------------------------------------------


def _gpu_step1(torch, ctx, kmx, pts4, prm, nbr_cap=None):
    p = dev(torch, pts4)
    grid = ctx.build_grid(p, prm.r_fpfh)
    cap = nbr_cap if nbr_cap is not None else len(pts4) * 200
    out = ctx.normals(grid, prm, cap)
    ctx.sync()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    res["grid"] = grid
    res["dev_points"] = p
    res["dev"] = out
    return res


def _sets_equal(o_offs, o_nbr, g_offs, g_nbr):
    assert np.array_equal(o_offs, g_offs)
    for q in range(len(o_offs) - 1):
        a = o_nbr[o_offs[q]:o_offs[q + 1]]
        b = np.sort(g_nbr[g_offs[q]:g_offs[q + 1]])
        if not np.array_equal(a, b):
            return q
    return -1


@pytest.mark.parametrize("case", ["scene", "lidar", "ties"])
def test_neighbour_sets_bit_exact(torch_cuda, ctx, orc, case):
    from paper_2409_15615_gb300 import kmx

    torch = torch_cuda
    if case == "scene":
        vs, _ = orc.voxelize(scene_pair(2)[0], 0.1)
        v = 0.1
    elif case == "lidar":
        vs, _ = orc.voxelize(lidar_pair(2)[0], 0.3)
        v = 0.3
    else:
        # a lattice of spacing 1/8 with r_FPFH = 0.5 exactly: many distances equal
        # the radius and must be excluded (strict < of Eq. A1)
        g = np.arange(-6, 7) * 0.125
        xx, yy, zz = np.meshgrid(g, g, g[:5])
        vs = np.stack([xx.ravel(), yy.ravel(), zz.ravel(), 0 * xx.ravel()], 1).astype(np.float32)
        v = 0.1
    prm, oprm = params_for(kmx, orc, v, (0, 0, 0))
    if case == "ties":
        prm.r_fpfh, prm.r_normal = 0.5, 0.375
        oprm.r_fpfh, oprm.r_normal = 0.5, 0.375
    offs, nbr = orc.radius_search(vs, oprm.r_fpfh)
    g = _gpu_step1(torch, ctx, kmx, vs, prm)
    assert int(g["needed"][0]) == len(nbr)
    bad = _sets_equal(offs, nbr, g["offs"], g["nbr"])
    assert bad < 0, "neighbour set of point %d differs" % bad


def _normal_bands(o_n4, o_ev, pts, vp, tau_lin):
    l1, l2, l3 = o_ev[:, 0], o_ev[:, 1], o_ev[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        degenerate = (l2 - l3) / np.where(l1 > 0, l1, 1) < 1e-2
        view = vp[None, :] - pts[:, :3].astype(np.float64)
        sign_ill = np.abs(np.sum(o_n4[:, :3] * view, 1)) / np.maximum(np.linalg.norm(view, axis=1), 1e-300) < 1e-4
    lin_band = np.abs(o_n4[:, 3] - tau_lin) < 1e-5
    return degenerate | sign_ill, lin_band


@pytest.mark.parametrize("case", ["scene", "lidar"])
def test_normals_parity(torch_cuda, ctx, orc, case):
    from paper_2409_15615_gb300 import kmx

    torch = torch_cuda
    if case == "scene":
        src, _, _, _, vp, _ = scene_pair(4)
        v = 0.1
    else:
        src, _, _, _, vp, _ = lidar_pair(4)
        v = 0.3
    vs, _ = orc.voxelize(src, v)
    prm, oprm = params_for(kmx, orc, v, vp)
    offs, nbr = orc.radius_search(vs, oprm.r_fpfh)
    o_n4, o_ev, o_fl, _ = orc.normals(vs, offs, nbr, oprm)
    g = _gpu_step1(torch, ctx, kmx, vs, prm)
    g_n4, g_fl = g["normal4"][: len(vs)], g["flags"][: len(vs)]
    # PCA reached: depends on integer counts only -> exact
    assert np.array_equal(g_fl & 4, o_fl & 4)
    ill, lin_band = _normal_bands(o_n4, o_ev, vs, oprm.viewpoint, oprm.tau_lin)
    pca = (o_fl & 4) > 0
    check = pca & ~ill & (o_ev[:, 0] > 0)
    a = g_n4[check, :3].astype(np.float64)
    a /= np.linalg.norm(a, axis=1, keepdims=True)  # FP32 rounding leaves |a| = 1 +- 1e-7
    b = o_n4[check, :3]
    ang = np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.sum(a * b, 1))
    assert ang.max() <= NORMAL_TOL_RAD, "max normal angle %.3g rad" % ang.max()
    assert np.abs(g_n4[check, 3] - o_n4[check, 3]).max() < 1e-5
    same_b = (g_fl & 1) == (o_fl & 1)
    assert np.all(same_b | lin_band | ill), "B differs outside the bands at %s" % np.nonzero(~(same_b | lin_band | ill))[0][:10]
    assert check.mean() > 0.5


def test_neighbour_capacity_error(torch_cuda, ctx, orc):
    from paper_2409_15615_gb300 import kmx

    torch = torch_cuda
    vs, _ = orc.voxelize(scene_pair(5, n=4000)[0], 0.1)
    prm, oprm = params_for(kmx, orc, 0.1, (5, 5, 5))
    offs, nbr = orc.radius_search(vs, oprm.r_fpfh)
    p = dev(torch, vs)
    grid = ctx.build_grid(p, prm.r_fpfh)
    out = ctx.normals(grid, prm, 10)
    with pytest.raises(kmx.KmxError) as e:
        ctx.sync()
    assert e.value.status == kmx.KMX_ECAPACITY
    assert int(out["needed"].item()) == len(nbr)
    # the lists were not written: every offset is 0, so the next stage reads
    # empty lists (no entry past the 10-entry buffer) and describes nothing
    assert np.all(out["offs"].cpu().numpy() == 0)
    res = ctx.fasterpfh(grid, prm, out["normal4"], out["flags"], out["offs"], out["nbr"])
    ctx.sync()
    assert int(res["n_valid"].item()) == 0
    # a grid cell smaller than r_FPFH is refused on the host
    small = ctx.build_grid(p, prm.r_fpfh * 0.5)
    with pytest.raises(kmx.KmxError) as e:
        ctx.normals(small, prm, len(nbr))
    assert e.value.status == kmx.KMX_EINVAL
    ctx.sync()


# ----------------------------------------------------------------------------
# Faster-PFH (Algorithm 1 step 2, Eqs. A2-A5), stage-isolated on oracle inputs
# ----------------------------------------------------------------------------


from parity_helpers import fpfh_allowance as _fpfh_allowance  # noqa: E402
from parity_helpers import hist_violation as _hist_close  # noqa: E402
from parity_helpers import spfh_allowance as _spfh_allowance  # noqa: E402


@pytest.mark.parametrize("case", ["scene", "lidar"])
def test_fasterpfh_stage_isolated(torch_cuda, ctx, orc, case):
    """Every SPFH and FPFH row is checked; rows that contain flip-prone pairs
    (per the oracle) get the exact extra allowance those flips can cause."""
    from paper_2409_15615_gb300 import kmx

    torch = torch_cuda
    if case == "scene":
        src, _, _, _, vp, _ = scene_pair(6)
        v = 0.1
    else:
        src, _, _, _, vp, _ = lidar_pair(6)
        v = 0.3
    vs, _ = orc.voxelize(src, v)
    prm, oprm = params_for(kmx, orc, v, vp)
    # oracle step 1, then the oracle's own step 2 / SPFH / FPFH on FP32-cast normals
    offs, nbr = orc.radius_search(vs, oprm.r_fpfh)
    n4, ev, fl, _ = orc.normals(vs, offs, nbr, oprm)
    n4_32 = n4.astype(np.float32)
    n4_in = n4_32.astype(np.float64)
    voffs, vnbr, J, fl2 = orc.valid_filter(offs, nbr, fl, oprm.tau_num)
    sp, npairs, margin, n_marg = orc.spfh(vs, n4_in, fl2, voffs, vnbr, H, with_margin=True, band=FEATURE_BAND)
    fp = orc.fpfh(vs, J, voffs, vnbr, sp)
    # GPU step 2 on the same inputs
    p = dev(torch, vs)
    grid = ctx.build_grid(p, prm.r_fpfh)
    flags = dev(torch, fl & 5)
    res = ctx.fasterpfh(grid, prm, dev(torch, n4_32), flags, dev(torch, offs), dev(torch, nbr.astype(np.int32)),
                        want_spfh=True)
    ctx.sync()
    nJ = int(res["n_valid"].item())
    gJ = res["valid"][:nJ].cpu().numpy()
    assert np.array_equal(gJ, J)
    assert np.array_equal(flags.cpu().numpy(), fl2)
    gsp = res["spfh"][: len(vs), :33].cpu().numpy().astype(np.float64)
    a_sp = _spfh_allowance(n_marg, npairs)
    v_sp = _hist_close(gsp, sp, a_sp)
    assert v_sp.max() <= 1.0, "SPFH off by %.3g x tolerance" % v_sp.max()
    clean = a_sp == 0
    assert _hist_close(gsp[clean], sp[clean]).max() <= 1.0 and clean.mean() > 0.9
    assert np.all(res["spfh"][: len(vs), 33:].cpu().numpy() == 0)
    gfp = res["desc"][:nJ, :33].cpu().numpy().astype(np.float64)
    a_fp = _fpfh_allowance(vs, J, voffs, vnbr, a_sp)
    v_fp = _hist_close(gfp, fp, a_fp)
    assert v_fp.max() <= 1.0, "FPFH off by %.3g x tolerance" % v_fp.max()
    assert np.all(res["desc"][:nJ, 33:].cpu().numpy() == 0)


# ----------------------------------------------------------------------------
# mutual matching, stage-isolated on oracle descriptors
# ----------------------------------------------------------------------------


def _gap_band(o_side):
    g1 = (o_side["d2p"] - o_side["d1p"]) / np.maximum(o_side["d2p"], 1e-300)
    g2 = (o_side["d2q"] - o_side["d1q"]) / np.maximum(o_side["d2q"], 1e-300)
    return g1 < GAP_BAND, g2 < GAP_BAND


def _pad36(F):
    out = np.zeros((len(F), 36), np.float32)
    out[:, :33] = F
    return out


def _check_match(torch, ctx, orc, FP, FQ, mode):
    FP32 = FP.astype(np.float32)
    FQ32 = FQ.astype(np.float32)
    A, side = orc.mutual_match(FP32.astype(np.float64), FQ32.astype(np.float64))
    corr, n_out = ctx.match(dev(torch, _pad36(FP32)), None, len(FP), dev(torch, _pad36(FQ32)), None, len(FQ),
                            mode=mode)
    ctx.sync()
    n = int(n_out.item())
    c = corr[:n].cpu().numpy()
    gi, gj = c[:, 0], c[:, 1]
    gd1, gd2 = c[:, 2].view(np.float32), c[:, 3].view(np.float32)
    bp, bq = _gap_band(side)
    ref = {(int(i), int(j)) for i, j in zip(A["i"], A["j"])}
    got = {(int(i), int(j)) for i, j in zip(gi, gj)}
    for (i, j) in ref ^ got:
        jj = side["nn_pq"][i]
        assert bp[i] or bq[jj] or bq[j], "pair (%d, %d) differs outside the gap band" % (i, j)
    assert np.all(np.diff(gi) > 0)
    # distances of the common pairs
    refd = {(int(i), int(j)): (d1, d2) for i, j, d1, d2 in zip(A["i"], A["j"], A["d1"], A["d2"])}
    for i, j, d1, d2 in zip(gi, gj, gd1, gd2):
        if (int(i), int(j)) in refd:
            r1, r2 = refd[(int(i), int(j))]
            assert abs(d1 - r1) <= 1e-4 * max(r1, 1e-3) + 1e-4
            if np.isfinite(r2):
                assert abs(d2 - r2) <= 1e-4 * max(r2, 1e-3) + 1e-4
    return len(ref), len(ref ^ got)


@pytest.mark.parametrize("shape", [(700, 1300), (1, 5), (129, 128), (4099, 3001)])
def test_match_fp32_random(torch_cuda, ctx, orc, shape):
    from paper_2409_15615_gb300 import kmx

    rng = np.random.default_rng(sum(shape))
    FP = rng.gamma(0.5, 20.0, (shape[0], 33))
    FQ = rng.gamma(0.5, 20.0, (shape[1], 33))
    k = min(shape) // 2  # plant k near-copies so that there are true matches
    FQ[:k] = FP[rng.permutation(shape[0])[:k]] + rng.normal(0, 0.5, (k, 33))
    n_ref, n_diff = _check_match(torch_cuda, ctx, orc, FP, FQ, kmx.MATCH_FP32_EXACT)
    assert n_diff <= max(1, n_ref // 100)


def test_match_fp32_on_oracle_descriptors(torch_cuda, ctx, orc):
    from paper_2409_15615_gb300 import kmx

    src, tgt, _, _, vps, vpt = scene_pair(7)
    fs = orc.faster_pfh(orc.voxelize(src, 0.1)[0], orc.OracleParams(0.1, viewpoint=vps))
    ft = orc.faster_pfh(orc.voxelize(tgt, 0.1)[0], orc.OracleParams(0.1, viewpoint=vpt))
    n_ref, n_diff = _check_match(torch_cuda, ctx, orc, fs["fpfh"], ft["fpfh"], kmx.MATCH_FP32_EXACT)
    assert n_ref > 100


def _noalloc_match(torch, kmx, FP32, FQ32):
    """kmx_match_noalloc: the register-prefetch tiled kernel, no sorting, no
    dimension skipping; same FP32 arithmetic per distance."""
    import ctypes

    lib = kmx.library()
    fn = lib.kmx_match_noalloc
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    fn.restype = ctypes.c_int
    fn.argtypes = [vp, vp, i64, vp, vp, vp, i64, vp, vp, i64, vp, vp]
    dp, dq = dev(torch, _pad36(FP32)), dev(torch, _pad36(FQ32))
    cap = min(len(FP32), len(FQ32))
    out = torch.zeros((cap, 4), dtype=torch.int32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    st = fn(vp(dp.data_ptr()), None, len(FP32), None, vp(dq.data_ptr()), None, len(FQ32), None, vp(out.data_ptr()),
            cap, vp(n_out.data_ptr()), vp(stream.cuda_stream))
    assert st == kmx.KMX_OK
    torch.cuda.synchronize()
    return out[: int(n_out.item())].cpu().numpy()


def test_match_fp32_sparse_ties_equals_dense_kernel(torch_cuda, ctx, orc):
    """Rows drawn from a few zero patterns (so the exact path regroups rows and
    skips all-zero dimensions of tile pairs), exact duplicate rows and columns
    and all-zero rows (ties in both directions, resolved by the original
    index): the exact path equals the unsorted dense kernel byte for byte,
    and the oracle up to the gap band."""
    from paper_2409_15615_gb300 import kmx

    torch = torch_cuda
    rng = np.random.default_rng(11)
    patterns = rng.random((40, 33)) < 0.3
    patterns[:, [5, 16, 27]] = True

    def rows(n):
        return rng.gamma(0.5, 20.0, (n, 33)) * patterns[rng.integers(0, len(patterns), n)]

    FP, FQ = rows(3000), rows(2600)
    k = 800
    src = rng.permutation(3000)[:k]
    FQ[1000:1000 + k] = FP[src] + rng.normal(0, 0.3, (k, 33)) * (FP[src] != 0)
    FQ[100:160] = FQ[40:100]  # duplicate columns
    FP[200:260] = FP[10:70]  # duplicate rows
    FP[5] = 0.0
    FQ[7] = 0.0
    FQ[8] = 0.0
    FP32, FQ32 = FP.astype(np.float32), FQ.astype(np.float32)
    corr, n_out = ctx.match(dev(torch, _pad36(FP32)), None, len(FP32), dev(torch, _pad36(FQ32)), None, len(FQ32),
                            mode=kmx.MATCH_FP32_EXACT)
    ctx.sync()
    got = corr[: int(n_out.item())].cpu().numpy()
    ref = _noalloc_match(torch, kmx, FP32, FQ32)
    assert len(got) > k // 2
    assert got.shape == ref.shape and np.array_equal(got, ref)
    _check_match(torch, ctx, orc, FP, FQ, kmx.MATCH_FP32_EXACT)


def test_match_residency_does_not_change_results(torch_cuda, ctx):
    """The exact matcher's residency (1 or 2 CTAs per SM, a scheduling
    choice) changes the number of tile-pair ranges, the segments and the
    order of the column atomics, never the correspondences; out-of-range
    values are rejected."""
    from paper_2409_15615_gb300 import kmx

    torch = torch_cuda
    rng = np.random.default_rng(23)
    patterns = rng.random((30, 33)) < 0.3
    FP = (rng.gamma(0.5, 20.0, (2900, 33)) * patterns[rng.integers(0, 30, 2900)]).astype(np.float32)
    FQ = (rng.gamma(0.5, 20.0, (2700, 33)) * patterns[rng.integers(0, 30, 2700)]).astype(np.float32)
    FQ[300:500] = FP[:200]  # exact duplicates: ties resolved by original index
    dp, dq = dev(torch, _pad36(FP)), dev(torch, _pad36(FQ))
    outs = []
    for res in (0, 1, 2, 1):
        ctx.set_match_residency(res)
        corr, n_out = ctx.match(dp, None, len(FP), dq, None, len(FQ), mode=kmx.MATCH_FP32_EXACT)
        ctx.sync()
        outs.append(corr[: int(n_out.item())].cpu().numpy())
    ctx.set_match_residency(0)
    assert len(outs[0]) >= 200
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    for bad in (-1, 3):
        with pytest.raises(kmx.KmxError):
            ctx.set_match_residency(bad)


def test_match_empty(torch_cuda, ctx):
    torch = torch_cuda
    from paper_2409_15615_gb300 import kmx

    d = torch.zeros((4, 36), device="cuda")
    corr, n = ctx.match(d, None, 0, d, None, 4, mode=kmx.MATCH_FP32_EXACT, cap=4)
    ctx.sync()
    assert int(n.item()) == 0


# ----------------------------------------------------------------------------
# the chained pipeline (voxelise -> ... -> match) against the oracle's chain
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("case", ["scene", "lidar", "scene_v005"])
def test_chained_pair(torch_cuda, ctx, orc, case):
    """The whole chain against the oracle.  Voxels bit-exact; J equal outside
    the points whose reliability (or a neighbour's) sits on the tau_lin band.
    The GPU's correspondences are then compared with the oracle's matching of
    the oracle's own FP64 step 2, SPFH and FPFH computed from the GPU's step-1
    outputs (normals and flags; neighbour lists are bit-exact): they must be
    equal except pairs attributed to a propagated band (a nearest-neighbour
    swap that the FP32 rounding of the descriptors, including pair features
    within 2e-6 of a decision edge, can cause: parity_helpers.attribute_pairs).
    The difference between that and the oracle's whole chain stems from the
    normals alone, which the normals tests hold to 1e-5 rad outside the
    ill-posed bands; its size is reported in the assertion messages."""
    from paper_2409_15615_gb300 import kmx, pipeline
    from parity_helpers import attribute_pairs, lin_bands, row_allowance

    torch = torch_cuda
    if case == "scene":
        src, tgt, R, t, vps, vpt = scene_pair(8)
        v = 0.1
    elif case == "scene_v005":
        src, tgt, R, t, vps, vpt = scene_pair(18, n=60000)
        v = 0.05
    else:
        src, tgt, R, t, vps, vpt = lidar_pair(8)
        v = 0.3
    vp_s, vp_t = np.float32(vps).astype(np.float64), np.float32(vpt).astype(np.float64)
    A, fs, ft, vs, vt = orc.front_end(src, tgt, v, vp_s, vp_t)
    ps, _ = params_for(kmx, orc, v, vps)
    pt, _ = params_for(kmx, orc, v, vpt)
    pair = pipeline.PairState(ctx, len(src), len(tgt))
    pair.src.raw.copy_(dev(torch, src))
    pair.tgt.raw.copy_(dev(torch, tgt))
    pair.run_checked(len(src), len(tgt), ps, pt, kmx.MATCH_FP32_EXACT)
    assert int(pair.src.n_vox.item()) == len(vs) and int(pair.tgt.n_vox.item()) == len(vt)
    assert np.array_equal(pair.src.vox4[: len(vs)].cpu().numpy().view(np.uint32), vs.view(np.uint32))
    assert np.array_equal(pair.tgt.vox4[: len(vt)].cpu().numpy().view(np.uint32), vt.view(np.uint32))
    hyb = []
    for cs, fo, pts in ((pair.src, fs, vs), (pair.tgt, ft, vt)):
        n = len(pts)
        _, j_band = lin_bands(pts, fo, 0.99)
        nJ = int(cs.out["n_valid"].item())
        gJ = cs.out["valid"][:nJ].cpu().numpy()
        diff = np.setxor1d(gJ, fo["J"])
        assert j_band[diff].all(), "J differs outside the tau_lin band at %s" % diff[~j_band[diff]][:10]
        # the oracle's step 2 and descriptors on the GPU's step-1 outputs
        n4g = cs.bufs["normal4"][:n].cpu().numpy().astype(np.float64)
        flg = cs.bufs["flags"][:n].cpu().numpy()
        voffs, vnbr, J, fl2 = orc.valid_filter(fo["offs"], fo["nbr"], flg & 5, 3)
        assert np.array_equal(J, gJ)
        sp, npairs, _, n_marg = orc.spfh(pts, n4g, fl2, voffs, vnbr, H, with_margin=True, band=FEATURE_BAND)
        F = orc.fpfh(pts, J, voffs, vnbr, sp)
        hyb.append((J, F, row_allowance(pts, J, voffs, vnbr, n_marg, npairs, F),
                    cs.out["desc"][:nJ, :33].cpu().numpy().astype(np.float64)))
    gi, gj, gd1, gd2 = pair.correspondences()
    pair.close()
    G = np.zeros(len(gi), dtype=A.dtype)
    G["i"], G["j"] = gi, gj
    (Jp, Fp, ap, gp), (Jq, Fq, aq, gq) = hyb
    # every row's measured deviation lies within its band; the swaps are then
    # attributed to the deviations that occurred
    dp = np.linalg.norm(gp - Fp, axis=1)
    dq = np.linalg.norm(gq - Fq, axis=1)
    assert np.all(dp <= ap) and np.all(dq <= aq), "a descriptor row deviates beyond its band"
    H_, _ = orc.mutual_match(Fp, Fq)
    Hp = H_.copy()
    Hp["i"], Hp["j"] = Jp[H_["i"]], Jq[H_["j"]]
    bad, why = attribute_pairs(Hp, G, Fp, Fq, Jp, Jq, gp, gq, Jp, Jq, dp, dq, orc.mutual_match)
    whole = len(set(zip(A["i"].tolist(), A["j"].tolist())) ^ set(zip(Hp["i"].tolist(), Hp["j"].tolist())))
    assert not bad, "pairs differ without a band: %s (%s; the normals move %d of %d pairs)" % (
        bad[:5], why, whole, len(A))
    assert why["pairs"] > 100, (why, whole)


# ----------------------------------------------------------------------------
# BF16 tensor-core candidates + exact FP32 re-ranking
# ----------------------------------------------------------------------------


def _gpu_match(torch, ctx, FP32, FQ32, mode):
    corr, n_out = ctx.match(dev(torch, _pad36(FP32)), None, len(FP32), dev(torch, _pad36(FQ32)), None, len(FQ32),
                            mode=mode)
    ctx.sync()
    c = corr[: int(n_out.item())].cpu().numpy()
    return c[:, 0], c[:, 1], c[:, 2].view(np.float32), c[:, 3].view(np.float32)


def _same_as_exact(torch, ctx, FP32, FQ32):
    """KMX_MATCH_BF16_RERANK must return exactly the bytes of
    KMX_MATCH_FP32_EXACT: the same pairs in the same order with the same d1
    and d2 (the candidates provably hold every column up to the second-nearest
    one, and they are re-ranked with the exact path's arithmetic)."""
    from paper_2409_15615_gb300 import kmx

    a = _gpu_match(torch, ctx, FP32, FQ32, kmx.MATCH_FP32_EXACT)
    b = _gpu_match(torch, ctx, FP32, FQ32, kmx.MATCH_BF16_RERANK)
    assert len(a[0]) == len(b[0]), "%d pairs against %d" % (len(b[0]), len(a[0]))
    for x, y, name in zip(a, b, ("i", "j", "d1", "d2")):
        assert np.array_equal(x.view(np.int32), y.view(np.int32)), "%s differs in %d rows" % (
            name, int(np.sum(x.view(np.int32) != y.view(np.int32))))
    return len(a[0])


@pytest.mark.parametrize("shape", [(700, 1300), (1, 5), (129, 128), (4099, 3001)])
def test_match_bf16_random(torch_cuda, ctx, orc, shape):
    from paper_2409_15615_gb300 import kmx

    rng = np.random.default_rng(sum(shape) + 1)
    FP = rng.gamma(0.5, 20.0, (shape[0], 33))
    FQ = rng.gamma(0.5, 20.0, (shape[1], 33))
    k = min(shape) // 2
    FQ[:k] = FP[rng.permutation(shape[0])[:k]] + rng.normal(0, 0.5, (k, 33))
    n_ref, n_diff = _check_match(torch_cuda, ctx, orc, FP, FQ, kmx.MATCH_BF16_RERANK)
    assert n_diff <= max(1, n_ref // 100)
    _same_as_exact(torch_cuda, ctx, FP.astype(np.float32), FQ.astype(np.float32))


def test_match_bf16_equals_exact_fp32(torch_cuda, ctx, orc):
    """On LiDAR-scan descriptors (plane-dominated: many near-duplicate rows),
    the tensor-core path returns the exact path's correspondences byte for
    byte, and almost every row is settled by its candidate list."""
    from paper_2409_15615_gb300 import kmx

    src, tgt, _, _, vps, vpt = lidar_pair(9)
    fs = orc.faster_pfh(orc.voxelize(src, 0.3)[0], orc.OracleParams(0.3, viewpoint=vps))
    ft = orc.faster_pfh(orc.voxelize(tgt, 0.3)[0], orc.OracleParams(0.3, viewpoint=vpt))
    FP, FQ = fs["fpfh"].astype(np.float32), ft["fpfh"].astype(np.float32)
    n = _same_as_exact(torch_cuda, ctx, FP, FQ)
    assert n > 1000
    diag = ctx.match_diag(len(FP), len(FQ)).cpu().numpy()
    assert diag[0] + diag[1] <= (len(FP) + len(FQ)) // 100, "fallback rows %s" % diag[:2]
    assert diag[2] >= 2 * len(FP) - 2 and diag[3] >= 2 * len(FQ) - 2


@pytest.mark.parametrize("clustered", [True, False])
def test_match_bf16_many_items(torch_cuda, ctx, clustered):
    """Sizes with several work items per row tile and several items per
    persistent CTA (row tiles change between a CTA's items): byte equality
    with the exact path.  On clustered descriptors (mixtures of tight
    clusters, like the near-duplicate rows of planes) the triangle-inequality
    test leaves only a part of the tile pairs to the tensor cores; on
    unstructured ones it may keep nearly all."""
    rng = np.random.default_rng(77 + clustered)
    if clustered:
        cen = rng.gamma(0.5, 20.0, (60, 33))
        FP = (cen[rng.integers(0, 60, 20000)] + rng.normal(0, 0.6, (20000, 33))).astype(np.float32)
        FQ = (cen[rng.integers(0, 60, 12000)] + rng.normal(0, 0.6, (12000, 33))).astype(np.float32)
    else:
        FP = rng.gamma(0.5, 20.0, (20000, 33)).astype(np.float32)
        FQ = rng.gamma(0.5, 20.0, (12000, 33)).astype(np.float32)
    n = _same_as_exact(torch_cuda, ctx, FP, FQ)
    assert n > 0
    d = ctx.match_diag(len(FP), len(FQ)).cpu().numpy()
    all_pairs = -(-len(FP) // 128) * -(-len(FQ) // 128)
    assert 0 < d[4] <= all_pairs and 0 < d[5] <= all_pairs
    if clustered:
        assert d[4] + d[5] < all_pairs, "pruning left %s of %d tile pairs" % (d[4:], 2 * all_pairs)


def test_match_bf16_duplicates_overflow_to_exact(torch_cuda, ctx):
    """600 copies of one descriptor tie at distance 0 for every row near them:
    those rows' candidate lists overflow (512) and go through the exact FP32
    tiles; ties resolve to the lowest index exactly as in the exact path."""
    rng = np.random.default_rng(21)
    FP = rng.gamma(0.5, 20.0, (900, 33)).astype(np.float32)
    FQ = rng.gamma(0.5, 20.0, (1100, 33)).astype(np.float32)
    FQ[100:700] = FP[5]
    FP[600:650] = FP[5]
    n = _same_as_exact(torch_cuda, ctx, FP, FQ)
    assert n > 0
    diag = ctx.match_diag(len(FP), len(FQ)).cpu().numpy()
    assert diag[0] >= 51, "the 51 rows equal to the duplicated descriptor overflow: %s" % diag


@pytest.mark.parametrize("overflow_rows", [64, 65, 201])
def test_match_bf16_overflow_row_counts(torch_cuda, ctx, overflow_rows):
    """overflow_rows source rows equal one descriptor that 600 target rows
    copy: all of them overflow.  Up to 64 listed rows the fallback streams
    each row over column chunks, above that it runs the tiled kernel; both
    sides of the switch give the exact path's bytes."""
    rng = np.random.default_rng(29)
    FP = rng.gamma(0.5, 20.0, (900, 33)).astype(np.float32)
    FQ = rng.gamma(0.5, 20.0, (3000, 33)).astype(np.float32)
    FQ[100:700] = FP[5]
    FP[600:600 + overflow_rows - 1] = FP[5]
    n = _same_as_exact(torch_cuda, ctx, FP, FQ)
    assert n > 0
    diag = ctx.match_diag(len(FP), len(FQ)).cpu().numpy()
    assert diag[0] >= overflow_rows, "overflowed rows: %s" % diag


def test_match_bf16_one_overflow_row_many_columns(torch_cuda, ctx):
    """One source row ties with 700 target rows: its list overflows and the
    exact fallback spreads that single row over hundreds of column chunks
    (partials packed by the list length); the result is byte-identical."""
    rng = np.random.default_rng(23)
    FP = rng.gamma(0.5, 20.0, (2000, 33)).astype(np.float32)
    FQ = rng.gamma(0.5, 20.0, (40000, 33)).astype(np.float32)
    FQ[1000:1700] = FP[7]
    n = _same_as_exact(torch_cuda, ctx, FP, FQ)
    assert n > 0
    diag = ctx.match_diag(len(FP), len(FQ)).cpu().numpy()
    assert diag[0] >= 1, "row 7 overflows: %s" % diag


def test_match_bf16_nonfinite_is_range_error(torch_cuda, ctx):
    from paper_2409_15615_gb300 import kmx

    FP = np.ones((300, 33), np.float32)
    FQ = np.ones((200, 33), np.float32)
    FP[17, 4] = np.nan
    ctx.match(dev(torch_cuda, _pad36(FP)), None, len(FP), dev(torch_cuda, _pad36(FQ)), None, len(FQ),
              mode=kmx.MATCH_BF16_RERANK)
    with pytest.raises(kmx.KmxError) as e:
        ctx.sync()
    assert e.value.status == kmx.KMX_ERANGE


def test_match_bf16_on_oracle_descriptors(torch_cuda, ctx, orc):
    from paper_2409_15615_gb300 import kmx

    src, tgt, _, _, vps, vpt = scene_pair(10)
    fs = orc.faster_pfh(orc.voxelize(src, 0.1)[0], orc.OracleParams(0.1, viewpoint=vps))
    ft = orc.faster_pfh(orc.voxelize(tgt, 0.1)[0], orc.OracleParams(0.1, viewpoint=vpt))
    n_ref, n_diff = _check_match(torch_cuda, ctx, orc, fs["fpfh"], ft["fpfh"], kmx.MATCH_BF16_RERANK)
    assert n_ref > 100
