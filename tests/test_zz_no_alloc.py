"""kmx_match_noalloc: the matching entry point for callers that cannot
allocate device memory while they match (a memory pool that already owns the
device, a real-time loop that may not block on the allocator, a host framework
that forbids allocation calls).  It must give the same correspondences as
kmx_match in exact FP32 mode, call after call, although every call reuses one
fixed scratch array.  Collected last on purpose (file name)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pad36(F):
    out = np.zeros((len(F), 36), np.float32)
    out[:, :33] = F
    return out


def test_noalloc_equals_kmx_match_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_15615_gb300 import build, kmx

    build.build()
    lib = kmx.library()
    fn = lib.kmx_match_noalloc
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    fn.restype = ctypes.c_int
    fn.argtypes = [vp, vp, i64, vp, vp, vp, i64, vp, vp, i64, vp, vp]
    ctx = kmx.Context(0)
    stream = torch.cuda.current_stream()

    def p(t):
        return None if t is None else vp(t.data_ptr())

    # two ordinary calls in a row, then one at the stated maximum on both
    # sides, where the fixed array's size actually binds
    top = kmx.KMX_NOALLOC_MAX_ROWS
    for trial, (n_p, n_q) in enumerate([(3000, 2500), (1200, 4100), (top, top)]):
        rng = np.random.default_rng(100 + trial)
        FP = rng.gamma(0.5, 20.0, (n_p, 33)).astype(np.float32)
        FQ = rng.gamma(0.5, 20.0, (n_q, 33)).astype(np.float32)
        k = min(n_p, n_q) // 2
        FQ[:k] = FP[rng.permutation(n_p)[:k]] + rng.normal(0, 0.5, (k, 33)).astype(np.float32)
        dp = torch.from_numpy(_pad36(FP)).cuda()
        dq = torch.from_numpy(_pad36(FQ)).cuda()
        # valid lists map rows to point ids: the emitted (i, j) go through them
        vpl = torch.arange(n_p, dtype=torch.int32, device="cuda") * 3 + 1
        vql = torch.arange(n_q, dtype=torch.int32, device="cuda") * 5 + 2
        ref, n_ref = ctx.match(dp, vpl, n_p, dq, vql, n_q, mode=kmx.MATCH_FP32_EXACT)
        ctx.sync()
        cap = min(n_p, n_q)
        out = torch.full((cap, 4), -7, dtype=torch.int32, device="cuda")
        n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = fn(p(dp), p(vpl), n_p, None, p(dq), p(vql), n_q, None, p(out), cap, p(n_out), vp(stream.cuda_stream))
        assert st == kmx.KMX_OK
        torch.cuda.synchronize()
        n = int(n_out.item())
        # -1 would report a prefix-scan wait that gave up
        assert n >= 0
        assert n == int(n_ref.item()) and n > k // 2
        a = ref[:n].cpu().numpy()
        b = out[:n].cpu().numpy()
        assert np.array_equal(a[:, :2], b[:, :2])
        assert np.allclose(a[:, 2:].view(np.float32), b[:, 2:].view(np.float32), rtol=1e-6, atol=0)
    # sizes beyond the stated maximum are refused without launching anything
    big = top + 1
    st = fn(p(dp), None, big, None, p(dq), None, 10, None, p(out), 10, p(n_out), vp(stream.cuda_stream))
    assert st == kmx.KMX_EINVAL
    ctx.close()
