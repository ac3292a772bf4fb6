"""The m = 2 records pipeline with its deep levels taken per group of ranks,
on the CPU (no GPU, no CUDA code): a plain Python model of what the library
computes when the levels below gS run in shared memory (k_group) and the
others through the records in HBM.

Levels lv < gS.  Records of level lv are keyed by the node r >> (lv+1)
(Sec. 5); all of them share the group r >> gS with their point, so the points
(in the order of the last coordinate, queries first on ties) are sorted
stably by group, and within a group the order of level lv-1 is the order of
level lv split stably by bit lv inside every node of level lv.  In that
order each level's records (data with bit lv = 0, queries with bit lv = 1)
are sorted by (node, last coordinate), so a segmented scan gives every query
F over the data of its node before it.

Levels lv >= gS.  The records of the level, in the order of the last
coordinate, sorted stably by node, then the same segmented scan.

The sum over all levels equals the definition (brute force) on random
inputs with heavy ties, for strict and non-strict first coordinates, and for
every gS from 0 (every level in HBM) to b (every level in groups)."""
import numpy as np
import pytest


def _ranks(P, nD, nonstrict0):
    _, r = np.unique(P[:, 0], return_inverse=True)
    r = r.astype(np.int64)
    if nonstrict0:  # d0 <= q0  <=>  2 r(d) < 2 r(q) + 1
        r = 2 * r + (np.arange(P.shape[0]) >= nD)
    return r


def _order_last(P, nD):
    isq = np.arange(P.shape[0]) >= nD
    return np.lexsort((~isq, P[:, 1]))  # queries first on a tie of the last coordinate


def _scan_level(seq, lv, r, isq, w, out):
    """Segmented scan of one level over the points `seq` (already in node
    order): queries with bit lv = 1 receive F over the preceding data with
    bit lv = 0 of the same node."""
    acc, prev = 0, None
    for i in seq:
        node = r[i] >> (lv + 1)
        if node != prev:
            acc, prev = 0, node
        bit = (r[i] >> lv) & 1
        if isq[i] and bit == 1:
            out[i] += acc
        elif not isq[i] and bit == 0:
            acc += w[i]


def _pipeline(D, Q, w, gS, nonstrict0=False):
    nD = D.shape[0]
    P = np.concatenate([D, Q])
    n = P.shape[0]
    isq = np.arange(n) >= nD
    r = _ranks(P, nD, nonstrict0)
    b = int(np.ceil(np.log2(r.max() + 1))) if n and r.max() > 0 else 0
    gS = min(gS, b)
    wfull = np.concatenate([w, np.zeros(len(Q), np.int64)])
    out = np.zeros(n, np.int64)
    xo = _order_last(P, nD)
    # levels >= gS: records in the order of the last coordinate, sorted stably by node
    for lv in range(gS, b):
        rec = [i for i in xo if ((r[i] >> lv) & 1) == (1 if isq[i] else 0)]
        rec.sort(key=lambda i: r[i] >> (lv + 1))  # Python's sort is stable
        _scan_level(rec, lv, r, isq, wfull, out)
    # levels < gS: per group, split level by level
    if gS > 0:
        grouped = sorted(xo, key=lambda i: r[i] >> gS)  # stable by group
        groups = {}
        for i in grouped:
            groups.setdefault(r[i] >> gS, []).append(i)
        for pts in groups.values():
            order = list(pts)
            for lv in range(gS - 1, -1, -1):
                _scan_level(order, lv, r, isq, wfull, out)
                # split every node of level lv by bit lv (stable)
                new, k = [], 0
                while k < len(order):
                    j = k
                    while j < len(order) and (r[order[j]] >> (lv + 1)) == (r[order[k]] >> (lv + 1)):
                        j += 1
                    node = order[k:j]
                    new += [i for i in node if not (r[i] >> lv) & 1] + [i for i in node if (r[i] >> lv) & 1]
                    k = j
                order = new
    return out[nD:]


def _brute(D, Q, w, nonstrict0=False):
    lt0 = (D[None, :, 0] <= Q[:, None, 0]) if nonstrict0 else (D[None, :, 0] < Q[:, None, 0])
    dom = lt0 & (D[None, :, 1] < Q[:, None, 1])
    return (dom * w[None, :]).sum(axis=1)


@pytest.mark.parametrize("nonstrict0", [False, True])
def test_group_levels_equal_definition(nonstrict0):
    rng = np.random.default_rng(2305 + nonstrict0)
    for _ in range(40):
        nD, nQ = int(rng.integers(0, 60)), int(rng.integers(1, 60))
        levels = int(rng.integers(1, 40))
        D = rng.integers(0, levels, size=(nD, 2))
        Q = rng.integers(0, levels, size=(nQ, 2))
        w = rng.integers(-9, 10, size=nD).astype(np.int64)
        want = _brute(D, Q, w, nonstrict0)
        for gS in range(0, 8):
            assert np.array_equal(_pipeline(D, Q, w, gS, nonstrict0), want), (gS, nD, nQ, levels)


def test_group_levels_hand_case():
    # ranks 0..3 (b = 2), one group of 4 ranks at gS = 2: level 1 splits the
    # group by bit 1; level 0 then sees nodes {0,1} and {2,3}
    D = np.array([[0, 0], [1, 2], [2, 1]])
    Q = np.array([[3, 3], [1, 3], [2, 2]])
    w = np.array([1, 10, 100], np.int64)
    want = _brute(D, Q, w)
    assert want.tolist() == [111, 1, 1]
    for gS in (0, 1, 2):
        assert _pipeline(D, Q, w, gS).tolist() == want.tolist()
