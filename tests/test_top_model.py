"""The m = 2 records pipeline with its levels split three ways, on the CPU
(no GPU, no CUDA code): a plain Python model of what the library computes
when the levels below gS run per group of ranks (k_group), the levels from
tS = max(gS, b - top_bits) up run per tile of points with node sums carried
across tiles and ranges of tiles (k_top, k_top_carry, k_reduce_top), and
the levels in between go through the records in HBM.

Top levels.  The points, in the order of the last coordinate (queries first
on ties), are cut into tiles, and consecutive tiles into ranges.  Inside a
tile, level lv's records are ordered by (node r >> (lv+1), last coordinate)
by splitting the tile level by level from the top; a node's scan starts
from F over the node's data in the range's earlier tiles (frun), and F at
the node's end in the tile becomes the new frun.  At a range's end the
nodes' F over the range (agg) are scanned over the instance's ranges in
order, and each query of a later range adds the carry of its node at every
top level where it has a record.  Each (datum, query) pair is thereby
counted once, at the highest rank bit where they differ (Lemma 1).

The sum equals the definition (brute force) on random inputs with heavy
ties for every split (gS, top_bits), tile and range size, and for a
non-strict first coordinate."""
import numpy as np
import pytest


def _ranks(P, nD, nonstrict0):
    _, r = np.unique(P[:, 0], return_inverse=True)
    r = r.astype(np.int64)
    if nonstrict0:  # d0 <= q0  <=>  2 r(d) < 2 r(q) + 1
        r = 2 * r + (np.arange(P.shape[0]) >= nD)
    return r


def _scan(seq, node_of, bit_of, isq, w, out, start=None, totals=None):
    """Segmented scan over `seq` (in node order): queries with bit 1 receive F
    over the preceding data with bit 0 of the same node, starting from
    start[node] (the node's earlier tiles); F at each node's end into
    totals[node]."""
    acc, prev = 0, None
    for i in seq:
        nd = node_of(i)
        if nd != prev:
            acc, prev = (start or {}).get(nd, 0), nd
        if isq[i] and bit_of(i) == 1:
            out[i] += acc
        elif not isq[i] and bit_of(i) == 0:
            acc += w[i]
        if totals is not None:
            totals[nd] = acc


def _split(order, node_of, bit_of):
    new, k = [], 0
    while k < len(order):
        j = k
        while j < len(order) and node_of(order[j]) == node_of(order[k]):
            j += 1
        run = order[k:j]
        new += [i for i in run if bit_of(i) == 0] + [i for i in run if bit_of(i) == 1]
        k = j
    return new


def _pipeline(D, Q, w, gS, top_bits, tile, range_tiles, nonstrict0=False):
    nD = D.shape[0]
    P = np.concatenate([D, Q])
    n = P.shape[0]
    isq = np.arange(n) >= nD
    r = _ranks(P, nD, nonstrict0)
    b = int(r.max()).bit_length() if n and r.max() > 0 else 0
    gS = min(gS, b)
    tS = max(gS, b - top_bits) if top_bits > 0 else b
    wf = np.concatenate([w, np.zeros(len(Q), np.int64)])
    out = np.zeros(n, np.int64)
    xo = list(np.lexsort((~isq, P[:, 1])))
    node = lambda lv: (lambda i: r[i] >> (lv + 1))
    bit = lambda lv: (lambda i: (r[i] >> lv) & 1)
    # levels [gS, tS): records in the order of the last coordinate, sorted stably by node
    for lv in range(gS, tS):
        rec = [i for i in xo if bit(lv)(i) == int(isq[i])]
        rec.sort(key=node(lv))
        _scan(rec, node(lv), bit(lv), isq, wf, out)
    # levels >= tS: tiles of the order of the last coordinate, ranges of tiles
    carry = {lv: {} for lv in range(tS, b)}  # F over the earlier ranges, per node
    tiles = [xo[a:a + tile] for a in range(0, n, tile)]
    for r0 in range(0, len(tiles), range_tiles):
        frun = {lv: {} for lv in range(tS, b)}
        for pts in tiles[r0:r0 + range_tiles]:
            order = list(pts)  # the top level's order: one node, the last coordinate
            for lv in range(b - 1, tS - 1, -1):
                tot = dict(frun[lv])
                _scan(order, node(lv), bit(lv), isq, wf, out, start=frun[lv], totals=tot)
                frun[lv] = tot
                order = _split(order, node(lv), bit(lv))
        # the range's queries add their nodes' carries from the earlier ranges,
        # then the range's node totals join the carries (in range order)
        for pts in tiles[r0:r0 + range_tiles]:
            for i in pts:
                if isq[i]:
                    for lv in range(tS, b):
                        if bit(lv)(i) == 1:
                            out[i] += carry[lv].get(node(lv)(i), 0)
        for lv in range(tS, b):
            for nd, v in frun[lv].items():
                carry[lv][nd] = carry[lv].get(nd, 0) + v
    # levels < gS: per group, split level by level
    if gS > 0:
        groups = {}
        for i in xo:
            groups.setdefault(r[i] >> gS, []).append(i)
        for pts in groups.values():
            order = list(pts)
            for lv in range(gS - 1, -1, -1):
                _scan(order, node(lv), bit(lv), isq, wf, out)
                order = _split(order, node(lv), bit(lv))
    return out[nD:]


def _brute(D, Q, w, nonstrict0=False):
    lt0 = (D[None, :, 0] <= Q[:, None, 0]) if nonstrict0 else (D[None, :, 0] < Q[:, None, 0])
    dom = lt0 & (D[None, :, 1] < Q[:, None, 1])
    return (dom * w[None, :]).sum(axis=1)


@pytest.mark.parametrize("nonstrict0", [False, True])
def test_top_levels_equal_definition(nonstrict0):
    rng = np.random.default_rng(2307 + nonstrict0)
    for _ in range(25):
        nD, nQ = int(rng.integers(0, 50)), int(rng.integers(1, 50))
        levels = int(rng.integers(1, 60))
        D = rng.integers(0, levels, size=(nD, 2))
        Q = rng.integers(0, levels, size=(nQ, 2))
        w = rng.integers(-9, 10, size=nD).astype(np.int64)
        want = _brute(D, Q, w, nonstrict0)
        for gS, top_bits in ((0, 0), (0, 3), (2, 2), (3, 12), (0, 12), (7, 1)):
            for tile, range_tiles in ((7, 1), (7, 3), (1000, 1)):
                got = _pipeline(D, Q, w, gS, top_bits, tile, range_tiles, nonstrict0)
                assert np.array_equal(got, want), (gS, top_bits, tile, range_tiles, nD, nQ, levels)


def test_top_levels_hand_case():
    """Eight points, ranks 0..3 (b = 2): with tiles of two points in ranges of
    one tile, every top-level node's F crosses tile and range boundaries."""
    D = np.array([[0, 0], [1, 2], [2, 1], [0, 3]])
    Q = np.array([[3, 3], [1, 3], [2, 2], [3, 1]])
    w = np.array([1, 10, 100, 1000], np.int64)
    want = _brute(D, Q, w)
    assert want.tolist() == [111, 1, 1, 1]
    for gS, top_bits in ((0, 2), (1, 1), (0, 1)):
        for tile, range_tiles in ((2, 1), (3, 2), (8, 1)):
            assert _pipeline(D, Q, w, gS, top_bits, tile, range_tiles).tolist() == want.tolist()
