"""Host logic of the batched form (CPU only): the longest-processing-time
assignment of pairs to lanes and the autotuner's coordinate search, the
latter with a stand-in runner whose times are given."""
import itertools

import numpy as np


def _makespan(queues, costs):
    return max(sum(costs[j] for j in q) for q in queues)


def test_lpt_assignment_partitions_and_bounds_the_makespan():
    from paper_2409_15615_gb300 import batch

    rng = np.random.default_rng(3)
    for trial in range(40):
        n = int(rng.integers(1, 9))
        lanes = int(rng.integers(1, 4))
        costs = rng.lognormal(0.0, 1.0, n).tolist()
        queues = batch._assign_lpt(costs, lanes)
        assert len(queues) == lanes
        flat = sorted(j for q in queues for j in q)
        assert flat == list(range(n)), "every pair exactly once"
        assert all(q == sorted(q) for q in queues), "a lane runs its pairs in index order"
        # brute force over every assignment: LPT stays within Graham's 4/3 - 1/(3m)
        best = min(_makespan([[j for j in range(n) if a[j] == k] for k in range(lanes)], costs)
                   for a in itertools.product(range(lanes), repeat=n))
        assert _makespan(queues, costs) <= (4.0 / 3.0 - 1.0 / (3 * lanes)) * best + 1e-12


def test_lpt_puts_the_largest_pairs_on_different_lanes():
    from paper_2409_15615_gb300 import batch

    queues = batch._assign_lpt([1.0, 100.0, 1.0, 90.0, 80.0, 1.0], 3)
    heads = sorted(max(q, key=lambda j: [1.0, 100.0, 1.0, 90.0, 80.0, 1.0][j]) for q in queues)
    assert heads == [1, 3, 4]


def test_autotune_coordinate_search(monkeypatch):
    """Lanes first (default chunks, no tensor-core pairs), then the chunk size
    at the best lane count, then the tensor-core size boundary at the best
    pair; the fastest runner is returned and every other one is closed."""
    from paper_2409_15615_gb300 import batch

    times = {(4, 0, None): 5.0, (8, 0, None): 3.0, (16, 0, None): 4.0,
             (8, 4, None): 3.5, (8, 16, None): 2.5,
             (8, 16, 1e10): 2.0, (8, 16, 4e10): 2.2, (8, 16, 1.6e11): 2.4}
    made = []

    class FakeRunner:
        def __init__(self, pairs, lanes, device, chunks, tc_min):
            self.key = (lanes, chunks, None if tc_min == float("inf") else tc_min)
            self.modes = [1 if tc_min != float("inf") else 0] * len(pairs)
            self.closed = False
            made.append(self)

        def prepare(self):
            return self

        def capture(self):
            pass

        def close(self):
            self.closed = True

    monkeypatch.setattr(batch, "BatchRunner", FakeRunner)
    monkeypatch.setattr(batch, "time_batch", lambda r, reps=3, graph=True: times[r.key])
    best, table = batch.autotune([object()] * 32)
    assert [(t["lanes"], t["chunks"], t["tc_min"]) for t in table] == list(times)
    assert best.key == (8, 16, 1e10) and not best.closed
    assert all(r.closed for r in made if r is not best)
    # lane counts above the number of pairs are skipped
    made.clear()
    best, table = batch.autotune([object()] * 6, lane_options=(4, 8), chunk_options=(), tc_options=(None,))
    assert [t["lanes"] for t in table] == [4] and best.key == (4, 0, None)
