"""Host logic of the serving loop (CPU only): admission by budget and
measured headroom, the request footprint estimate, the Poisson arrivals and
the latency statistics."""
import numpy as np


def test_admission_rule():
    from paper_2409_15615_gb300.serve import admissible

    G = 1 << 30
    # nothing in flight: always admitted, even above the budget or headroom
    assert admissible(100 * G, 0, 60 * G, 0, 2 * G)
    # within budget and headroom
    assert admissible(1 * G, 10 * G, 60 * G, 50 * G, 2 * G)
    # exactly at the budget is allowed; one byte over is not
    assert admissible(10 * G, 50 * G, 60 * G, 100 * G, 2 * G)
    assert not admissible(10 * G + 1, 50 * G, 60 * G, 100 * G, 2 * G)
    # the measured headroom must cover the request and the reserve
    assert admissible(1 * G, 1, 60 * G, 3 * G, 2 * G)
    assert not admissible(1 * G, 1, 60 * G, 3 * G - 1, 2 * G)


def test_request_bytes_grows_with_the_scan_and_the_map():
    from paper_2409_15615_gb300 import serve

    class M:
        def __init__(self, n_valid):
            self.n_valid = n_valid

    def req(n):
        return serve.Request(rid=0, map_id=0, xyz=np.zeros((n, 3), np.float32), voxel=0.1)

    a = serve.request_bytes(req(1000), M(5000))
    b = serve.request_bytes(req(2000), M(5000))
    c = serve.request_bytes(req(2000), M(9000))
    assert serve.BYTES_FIXED < a < b < c
    # per query point at least the lists (4 bytes an entry), the Faster-PFH
    # scratch (8 bytes an entry) and a descriptor row
    per_point = (b - a) / 1000
    assert per_point >= 12 * 96 + 4 * 36


def test_poisson_arrivals_and_latency_stats():
    from paper_2409_15615_gb300 import serve

    t = serve.poisson_arrivals(500.0, 20000, seed=1)
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 500.0) < 15.0  # mean rate within 3 %

    class R:
        def __init__(self, arrival, done):
            self.arrival, self.done = arrival, done

    done = [R(i * 0.01, i * 0.01 + 0.002 * (1 + (i % 10 == 9) * 9)) for i in range(100)]
    st = serve.latency_stats(done)
    assert st["n"] == 100
    assert abs(st["p50_ms"] - 2.0) < 1e-9
    assert 2.0 < st["p99_ms"] <= 20.0 + 1e-9
    assert abs(st["pairs_per_s"] - 100 / (done[-1].done - done[0].arrival)) < 1e-9
    assert serve.latency_stats([])["n"] == 0
