"""pipeline.PairStream: pairs streamed from pinned host memory with uploads
and downloads overlapping the neighbouring pairs' kernels give, pair for
pair, the correspondences of a plain PairState run on the same clouds."""
import numpy as np
import pytest

from synth import scene_pair

pytestmark = pytest.mark.gpu


def _pairs(k, n=8000):
    out = []
    for seed in range(k):
        src, tgt, _, _, vps, vpt = scene_pair(600 + seed, n=n, clutter=True)
        m = min(len(src), len(tgt), 6000)
        out.append((np.ascontiguousarray(src[:m]), np.ascontiguousarray(tgt[:m]), vps, vpt))
    return out


@pytest.mark.parametrize("graph,concurrent,slots", [(True, False, 2), (False, False, 2), (True, True, 2),
                                                   (True, True, 3), (False, True, 4), (True, True, 1)])
def test_stream_equals_plain_runs(graph, concurrent, slots):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_15615_gb300 import build, kmx, pipeline

    build.build()
    ctx = kmx.Context(0)
    pairs = _pairs(4)
    n = len(pairs[0][0])
    assert all(len(p[0]) == n and len(p[1]) == n for p in pairs)
    prm = kmx.params_default(0.1, viewpoint=np.float32(pairs[0][2]).tolist())
    # reference: each pair alone through PairState
    ref = []
    plain = pipeline.PairState(ctx, n, n)
    for src, tgt, _, _ in pairs:
        plain.src.raw.copy_(torch.from_numpy(src).cuda())
        plain.tgt.raw.copy_(torch.from_numpy(tgt).cuda())
        plain.run_checked(n, n, prm, prm, kmx.MATCH_FP32_EXACT)
        i, j, _, _ = plain.correspondences()
        ref.append(set(zip(i.tolist(), j.tolist())))
    plain.close()
    st = pipeline.PairStream(ctx, n, n, concurrent=concurrent, slots=slots)
    st.prepare(n, n, prm, prm, kmx.MATCH_FP32_EXACT, graph=graph, sample=(pairs[0][0], pairs[0][1]))
    hosts = [(torch.from_numpy(s).pin_memory(), torch.from_numpy(t).pin_memory()) for s, t, _, _ in pairs]
    outs = [(torch.empty(st.slots[0].corr.shape, dtype=torch.int32).pin_memory(),
             torch.empty(1, dtype=torch.int64).pin_memory()) for _ in range(8)]
    evs = []
    for k in range(8):  # each pair twice; with 2 or 3 slots every pair lands on two slots
        hs, ht = hosts[k % 4]
        evs.append(st.submit(hs, ht, outs[k][0], outs[k][1]))
    for ev in evs:
        ev.synchronize()
    st.sync()
    for k in range(8):
        c = outs[k][0][: int(outs[k][1][0])].numpy()
        assert set(zip(c[:, 0].tolist(), c[:, 1].tolist())) == ref[k % 4], "pair %d differs" % k
    st.close()
    ctx.close()
