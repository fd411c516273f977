"""Host model of the exact matcher's work split (match_fp32_bulk.cu).

The (row tile x column tile) grid, W = npt * nqt tile pairs flattened
row-major, is cut into chunks of consecutive pairs that CTAs take from a
counter: NA chunks of LA = max(4, ceil(W / (8 * ctas))) pairs, then the
last W - NA * LA pairs (about one large chunk per CTA) in chunks of
LB = max(4, ceil(that / (4 * ctas))) pairs, so that the CTAs finish
within a small chunk of each other.  The segment of chunk c in row tile rt
sits in slot c + rt of a ((8 + 4) * ctas + 1 + npt) * 128 array, and
merge_segments reads the chunks chunk_of(rt * nqt) .. chunk_of(rt * nqt +
nqt - 1) of row tile rt.  These checks pin that arithmetic for any order in
which the CTAs take the chunks: every tile pair is covered exactly once,
slots are unique and in bounds, and the merge reads exactly the segments
written for its row tile.
"""
import random

TILE = 128
CHUNKS_PER_CTA = 8
TAIL_CHUNKS_PER_CTA = 4
MIN_CHUNK = 4


def chunk_geo(W, ctas):
    per = CHUNKS_PER_CTA * ctas
    LA = max(MIN_CHUNK, -(-W // per))
    NA = (W - min(W, ctas * LA)) // LA
    WA = NA * LA
    LB = max(MIN_CHUNK, -(-(W - WA) // (TAIL_CHUNKS_PER_CTA * ctas)))
    NC = NA + -(-(W - WA) // LB)
    return dict(LA=LA, NA=NA, WA=WA, LB=LB, NC=NC)


def chunk_start(g, c):
    return c * g["LA"] if c < g["NA"] else g["WA"] + (c - g["NA"]) * g["LB"]


def chunk_len(g, c):
    return g["LA"] if c < g["NA"] else g["LB"]


def chunk_of(g, x):
    return x // g["LA"] if x < g["WA"] else g["NA"] + (x - g["WA"]) // g["LB"]


def _check(n_p, n_q, ctas):
    npt, nqt = -(-n_p // TILE), -(-n_q // TILE)
    W = npt * nqt
    if W == 0:
        return
    g = chunk_geo(W, ctas)
    NC = g["NC"]
    assert NC <= (CHUNKS_PER_CTA + TAIL_CHUNKS_PER_CTA) * ctas
    assert g["LA"] >= MIN_CHUNK and g["LB"] >= MIN_CHUNK and g["LB"] <= g["LA"]
    slots = {}
    covered = [0] * W
    for c in range(NC):  # the CTA that takes a chunk does not change what it writes
        L = chunk_len(g, c)
        for o in range(L):
            x = chunk_start(g, c) + o
            if x >= W:
                break
            assert chunk_of(g, x) == c
            covered[x] += 1
            rt, ct = divmod(x, nqt)
            if o == L - 1 or ct + 1 == nqt:  # segment end, as in the kernel
                key = c + rt
                assert key not in slots
                assert key < (CHUNKS_PER_CTA + TAIL_CHUNKS_PER_CTA) * ctas + 1 + npt
                slots[key] = (c, rt)
    assert covered == [1] * W
    # only the last chunk may be cut short by W
    for c in range(NC - 1):
        assert chunk_start(g, c) + chunk_len(g, c) == chunk_start(g, c + 1)
    for rt in range(npt):
        cf, cl = chunk_of(g, rt * nqt), chunk_of(g, rt * nqt + nqt - 1)
        assert [slots[c + rt] for c in range(cf, cl + 1)] == [(c, rt) for c in range(cf, cl + 1)]


def test_chunks_cover_every_tile_once():
    cases = [(1, 1, 304), (1, 5, 304), (129, 128, 304), (4099, 3001, 304), (12778, 12776, 304),
             (128, 121000, 304), (121000, 128, 304), (700, 1300, 152), (5, 5, 1), (0, 10, 304),
             (300000, 300000, 304)]
    rng = random.Random(0)
    cases += [(rng.randint(1, 30000), rng.randint(1, 30000), rng.choice([1, 2, 7, 152, 304, 456]))
              for _ in range(200)]
    for n_p, n_q, ctas in cases:
        _check(n_p, n_q, ctas)
