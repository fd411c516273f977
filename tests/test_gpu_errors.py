"""Error paths of the C ABI on the GPU: bounded waits report KMX_ETIMEOUT and
leave the context usable; bad arguments are refused on the host with
KMX_EINVAL before anything is launched.  Nothing here faults or traps."""
import ctypes

import numpy as np
import pytest

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


def test_bounded_wait_times_out_and_context_survives(env):
    torch, kmx, ctx = env
    ctx.check_timeout(20000)
    with pytest.raises(kmx.KmxError) as e:
        ctx.sync()
    assert e.value.status == kmx.KMX_ETIMEOUT
    # the error was cleared and the context still works
    x = torch.rand((1000, 3), device="cuda")
    out4, n_out, _ = ctx.voxelize(x, 0.1)
    ctx.sync()
    assert int(n_out.item()) > 0
    with pytest.raises(kmx.KmxError) as e:
        ctx.check_timeout(0)
    assert e.value.status == kmx.KMX_EINVAL


def test_bad_arguments_are_refused(env):
    torch, kmx, ctx = env
    lib = kmx.library()
    x = torch.rand((100, 5), device="cuda")
    with pytest.raises(kmx.KmxError) as e:
        ctx.voxelize(x, 0.1)  # stride 5
    assert e.value.status == kmx.KMX_EINVAL
    with pytest.raises(kmx.KmxError):
        ctx.voxelize(torch.rand((100, 3), device="cuda"), -1.0)
    # misaligned output rows
    buf = torch.empty(4 * 101 + 1, dtype=torch.float32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = lib.kmx_voxelize(ctx.h, ctypes.c_void_p(x.data_ptr()), 100, 3, ctypes.c_float(0.1),
                          ctypes.c_void_p(buf.data_ptr() + 4), 100, ctypes.c_void_p(n_out.data_ptr()), None)
    assert st == kmx.KMX_EINVAL
    pts = torch.rand((500, 4), device="cuda")
    prm = kmx.params_default(0.1)
    grid = ctx.build_grid(pts, prm.r_fpfh)
    bad = kmx.params_default(0.1)
    bad.r_normal = bad.r_fpfh * 2
    with pytest.raises(kmx.KmxError) as e:
        ctx.normals(grid, bad, 500 * 64)
    assert e.value.status == kmx.KMX_EINVAL
    bad = kmx.params_default(0.1)
    bad.hist_bins = 8
    with pytest.raises(kmx.KmxError):
        ctx.normals(grid, bad, 500 * 64)
    # a grid cannot be rebuilt over more points than its capacity
    with pytest.raises(kmx.KmxError) as e:
        ctx.build_grid(torch.rand((900, 4), device="cuda"), prm.r_fpfh, reuse=grid)
    assert e.value.status == kmx.KMX_EINVAL
    d = torch.zeros((10, 36), device="cuda")
    with pytest.raises(kmx.KmxError):
        ctx.match(d, None, 10, d, None, 10, mode=9)
    ctx.sync()


def test_match_capacity_overflow_is_reported(env):
    torch, kmx, ctx = env
    rng = np.random.default_rng(0)
    F = rng.random((200, 36)).astype(np.float32)
    F[:, 33:] = 0
    d = torch.from_numpy(F).cuda()
    corr, n = ctx.match(d, None, 200, d, None, 200, mode=kmx.MATCH_FP32_EXACT, cap=5)
    with pytest.raises(kmx.KmxError) as e:
        ctx.sync()
    assert e.value.status == kmx.KMX_ECAPACITY
    assert int(n.item()) == 200  # identical sets: every row is its own mutual neighbour


def test_match_non_finite_descriptor_is_reported(env):
    torch, kmx, ctx = env
    rng = np.random.default_rng(1)
    for bad in (np.nan, np.inf, -np.inf):
        F = rng.random((300, 36)).astype(np.float32)
        F[:, 33:] = 0
        G = F.copy()
        G[123, 7] = bad
        dp, dq = torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda()
        ctx.match(dp, None, 300, dq, None, 300, mode=kmx.MATCH_FP32_EXACT)
        with pytest.raises(kmx.KmxError) as e:
            ctx.sync()
        assert e.value.status == kmx.KMX_ERANGE
    # the context is still usable
    corr, n = ctx.match(dp, None, 300, dp, None, 300, mode=kmx.MATCH_FP32_EXACT)
    ctx.sync()
    assert int(n.item()) == 300


def test_context_after_a_device_error_gives_a_fresh_contexts_results(env):
    """After a recorded device error kmx_sync re-zeroes the context's scan
    status area; a whole pair (voxelise, grid, normals, Faster-PFH, match,
    every stage with its scans) then gives exactly what a fresh context
    gives."""
    torch, kmx, ctx = env
    from paper_2409_15615_gb300 import pipeline
    from synth import scene_pair

    src, tgt, _, _, vps, vpt = scene_pair(77, n=6000, clutter=True)
    prm_s = kmx.params_default(0.1, viewpoint=np.float32(vps).tolist())
    prm_t = kmx.params_default(0.1, viewpoint=np.float32(vpt).tolist())

    def run(c):
        st = pipeline.PairState(c, len(src), len(tgt), overlap=False)
        st.src.raw.copy_(torch.from_numpy(np.ascontiguousarray(src)).cuda())
        st.tgt.raw.copy_(torch.from_numpy(np.ascontiguousarray(tgt)).cuda())
        st.run_checked(len(src), len(tgt), prm_s, prm_t, kmx.MATCH_FP32_EXACT)
        i, j, _, _ = st.correspondences()
        st.close()
        return i, j

    fresh = kmx.Context(0)
    ref = run(fresh)
    fresh.close()
    ctx.check_timeout(20000)
    with pytest.raises(kmx.KmxError) as e:
        ctx.sync()
    assert e.value.status == kmx.KMX_ETIMEOUT
    got = run(ctx)
    assert len(ref[0]) > 100
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
