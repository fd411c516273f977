"""Host model of the exact matcher's work split (match_fp32_bulk.cu).

The (row tile x column tile) grid, W = npt * nqt tiles flattened row-major,
is split over G = min(ctas, W) CTAs: CTA b takes tiles [b W / G, (b+1) W / G).
A CTA writes one row-summary segment per row tile it touches, in slot b + rt;
merge_segments finds the CTAs that touched row tile rt in closed form,
b = floor(((x + 1) G - 1) / W) for the first and last tile x of the row tile.
These checks pin that arithmetic: every tile is covered exactly once, slots
are unique and inside the (ctas + npt) * 128 segment array, and the merge
visits exactly the CTAs that touched each row tile, in column order.
"""
import random

TILE = 128


def _check(n_p, n_q, ctas):
    npt, nqt = -(-n_p // TILE), -(-n_q // TILE)
    W = npt * nqt
    if W == 0:
        return
    G = min(ctas, W)
    slots = {}
    covered = [0] * W
    for b in range(G):
        w0, w1 = b * W // G, (b + 1) * W // G
        assert w1 - w0 >= 1
        rt = w0 // nqt
        for t in range(w1 - w0):
            w = w0 + t
            covered[w] += 1
            assert w // nqt == rt
            if t + 1 == w1 - w0 or (w + 1) % nqt == 0:
                key = b + rt
                assert key not in slots and key < ctas + npt
                slots[key] = (b, rt)
                rt += 1
    assert covered == [1] * W
    for rt in range(npt):
        x0, x1 = rt * nqt, rt * nqt + nqt - 1
        bf, bl = ((x0 + 1) * G - 1) // W, ((x1 + 1) * G - 1) // W
        touched = [b for b in range(G) if max(b * W // G, x0) < min((b + 1) * W // G, x1 + 1)]
        assert touched == list(range(bf, bl + 1))
        assert [slots[b + rt] for b in touched] == [(b, rt) for b in touched]


def test_split_covers_every_tile_once():
    cases = [(1, 1, 304), (1, 5, 304), (129, 128, 304), (4099, 3001, 304), (12778, 12776, 304),
             (128, 121000, 304), (121000, 128, 304), (700, 1300, 152), (5, 5, 1), (0, 10, 304)]
    rng = random.Random(0)
    cases += [(rng.randint(1, 30000), rng.randint(1, 30000), rng.choice([1, 2, 7, 152, 304, 456]))
              for _ in range(300)]
    for n_p, n_q, ctas in cases:
        _check(n_p, n_q, ctas)
