"""Batched (one CUDA-graph launch over many uneven pairs) and serving
(continuous batching against resident maps) forms give exactly the results of
the one-pair-at-a-time path."""
import numpy as np
import pytest

from synth import lidar_pair, scene_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_15615_gb300 import build

    build.build()
    return torch


def _single(torch, spec, mode):
    from paper_2409_15615_gb300 import kmx, pipeline

    ctx = kmx.Context(0)
    st = pipeline.PairState(ctx, len(spec.src), len(spec.tgt))
    st.src.raw.copy_(torch.from_numpy(spec.src).cuda())
    st.tgt.raw.copy_(torch.from_numpy(spec.tgt).cuda())
    ps = kmx.params_default(spec.voxel, viewpoint=np.float32(spec.vp_src).tolist())
    pt = kmx.params_default(spec.voxel, viewpoint=np.float32(spec.vp_tgt).tolist())
    st.run_checked(len(spec.src), len(spec.tgt), ps, pt, mode)
    out = st.correspondences()
    st.close()
    ctx.close()
    return out


def _specs():
    from paper_2409_15615_gb300.batch import PairSpec

    specs = []
    for k, n in enumerate([1500, 4000, 9000, 2500, 12000]):
        s, t, R, tt, vps, vpt = scene_pair(200 + k, n=n)
        specs.append(PairSpec(s, t, (0.1, 0.15, 0.1, 0.2, 0.1)[k], tuple(vps), tuple(vpt)))
    s, t, R, tt, vps, vpt = lidar_pair(210, az_bins=256)
    specs.append(PairSpec(s, t, 0.3, tuple(vps), tuple(vpt)))
    return specs


@pytest.mark.parametrize("mode,chunks,tc_min", [(0, 0, None), (1, 0, None), (0, 4, 5e7), (0, 16, 1.5e8)])
def test_batch_graph_equals_single_pairs(torch_cuda, mode, chunks, tc_min):
    """Every configuration the autotuner can pick (lanes, the exact matcher's
    chunk size, the size bucket that goes to the tensor-core matcher) gives
    the one-pair-at-a-time correspondences, replay after replay."""
    torch = torch_cuda
    from paper_2409_15615_gb300.batch import BatchRunner

    specs = _specs()
    ref = [_single(torch, sp, mode) for sp in specs]
    r = BatchRunner(specs, lanes=3, mode=mode, chunks=chunks, tc_min=tc_min).prepare()
    if tc_min is not None:
        assert 0 < sum(m != 0 for m in r.modes) < len(specs)
    r.capture()
    for rep in range(2):  # the graph replays to the same result
        r.corr.fill_(-1)
        r.n_corr.zero_()
        r.replay()
        torch.cuda.synchronize()
        got = r.results()
        for k in range(len(specs)):
            for a, b in zip(ref[k], got[k]):
                assert np.array_equal(a, b), "pair %d differs (replay %d)" % (k, rep)
        assert sum(len(g[0]) for g in got) > 50
    r.close()


def test_serving_alone_equals_in_the_mix(torch_cuda):
    """Continuous batching: requests admitted while others are in flight give
    the same correspondences as the same requests served one at a time."""
    torch = torch_cuda
    from paper_2409_15615_gb300 import kmx
    from paper_2409_15615_gb300.serve import Request, ResidentMap, Server, latency_stats

    ctx = kmx.Context(0)
    maps = []
    for k in range(2):
        xyz, _, _, _, vp, _ = scene_pair(300 + k, n=30000)
        maps.append(ResidentMap(ctx, xyz, 0.1, vp))
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(10):
        n = int(rng.integers(2000, 12000))
        q, _, _, _, vp, _ = scene_pair(400 + i, n=n)
        reqs.append(Request(rid=i, map_id=i % 2, xyz=q, voxel=0.1, viewpoint=tuple(vp), arrival=0.0))
    alone = {}
    for r in reqs:
        s1 = Server(maps, slots=1)
        d = s1.run([Request(r.rid, r.map_id, r.xyz, r.voxel, r.viewpoint, 0.0)], realtime=False)
        alone[r.rid] = d[0].corr
    mix = Server(maps, slots=4).run(reqs, realtime=False)
    assert len(mix) == len(reqs)
    for r in mix:
        assert np.array_equal(r.corr, alone[r.rid]), "request %d differs in the mix" % r.rid
    st = latency_stats(mix)
    assert st["n"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    # admission by free HBM: a reserve larger than the device holds still
    # admits one request at a time, and every request completes
    huge = Server(maps, slots=4, reserve_bytes=1 << 50)
    done = huge.run([Request(r.rid, r.map_id, r.xyz, r.voxel, r.viewpoint, 0.0) for r in reqs[:4]], realtime=False)
    assert len(done) == 4 and huge.stats["held_by_memory"] > 0
    for r in done:
        assert np.array_equal(r.corr, alone[r.rid])
    # admission by budget: with room for one request at a time they still all complete
    tight = Server(maps, slots=4, budget_bytes=1).run(
        [Request(r.rid, r.map_id, r.xyz, r.voxel, r.viewpoint, 0.0) for r in reqs[:4]], realtime=False)
    assert len(tight) == 4
    ctx.close()
