"""Host model of the exact matcher's work split (match_fp32_bulk.cu).

The (row tile x column tile) grid, W = npt * nqt tile pairs flattened
row-major, is cut into NC chunks of L consecutive pairs, with
L = max(4, ceil(W / (8 * ctas))); CTAs take chunks from a counter.  The
segment of chunk c in row tile rt sits in slot c + rt of a
(8 * ctas + 1 + npt) * 128 array, and merge_segments reads the chunks
floor(rt * nqt / L) .. floor((rt * nqt + nqt - 1) / L) of row tile rt.
These checks pin that arithmetic for any order in which the CTAs take the
chunks: every tile pair is covered exactly once, slots are unique and in
bounds, and the merge reads exactly the segments written for its row tile.
"""
import random

TILE = 128
CHUNKS_PER_CTA = 8
MIN_CHUNK = 4


def chunk_geo(W, ctas):
    per = CHUNKS_PER_CTA * ctas
    L = max(MIN_CHUNK, -(-W // per))
    return L, -(-W // L)


def _check(n_p, n_q, ctas):
    npt, nqt = -(-n_p // TILE), -(-n_q // TILE)
    W = npt * nqt
    if W == 0:
        return
    L, NC = chunk_geo(W, ctas)
    assert NC <= CHUNKS_PER_CTA * ctas and L > 3
    slots = {}
    covered = [0] * W
    for c in range(NC):  # the CTA that takes a chunk does not change what it writes
        for o in range(L):
            x = c * L + o
            if x >= W:
                break
            covered[x] += 1
            rt, ct = divmod(x, nqt)
            if o == L - 1 or ct + 1 == nqt:  # segment end, as in the kernel
                key = c + rt
                assert key not in slots and key < CHUNKS_PER_CTA * ctas + 1 + npt
                slots[key] = (c, rt)
    assert covered == [1] * W
    for rt in range(npt):
        cf, cl = rt * nqt // L, (rt * nqt + nqt - 1) // L
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
