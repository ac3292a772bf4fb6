"""The m = 3 records pipeline with its deep first-rank levels taken per group
of ranks, on the CPU (no GPU, no CUDA code): a plain Python model of what
the library computes when the levels below gS run in shared memory
(k_group3) and the others through the records in HBM.

A record of first-rank level lv and second-rank level j is keyed by the
node (r0 >> (lv+1), r1 >> (j+1)) (Sec. 5 with two bitstring coordinates);
a point emits it when its rank bits select it (data: bit lv of r0 = 0 and
bit j of r1 = 0; queries: both 1).  In the order of the last coordinate
(queries first on ties) sorted stably by key, a segmented scan gives every
query F over the data of its node before it.

Levels lv < gS, per group r0 >> gS (k_group3): the group's points are kept
in the order (r0 >> (lv+1), last coordinate) by one stable split per level;
level lv's emitting points are compacted in that order into blocks (runs of
one r0 >> (lv+1)), and the second rank's levels are walked over them with
the points' dense ranks among the group's second ranks: per level j a
segmented scan over the nodes (block, local rank >> (j+1)), then a stable
split by bit j.  At a level whose blocks hold at most `pair_max` points,
each query the level emits takes F directly over the earlier data of its
block (in that order) with a smaller second rank instead.  A group with
more than `cap` points (heavy ties) sends its points' records of those
levels through the HBM path instead.

The sum over all levels equals the definition (brute force) on random
inputs with heavy ties, for every gS and capacity, and for non-strict
first and second coordinates."""
import numpy as np
import pytest


def _ranks(x, nD, nonstrict):
    _, r = np.unique(x, return_inverse=True)
    r = r.astype(np.int64)
    if nonstrict:  # d <= q  <=>  2 r(d) < 2 r(q) + 1
        r = 2 * r + (np.arange(x.shape[0]) >= nD)
    return r


def _bits(r):
    return int(r.max()).bit_length() if r.size and r.max() > 0 else 0


def _scan(seq, node_of, bit_of, isq, w, out):
    """Segmented scan over `seq` (in node order): queries with bit 1 receive F
    over the preceding data with bit 0 of the same node."""
    acc, prev = 0, None
    for i in seq:
        nd = node_of(i)
        if nd != prev:
            acc, prev = 0, nd
        if isq[i] and bit_of(i) == 1:
            out[i] += acc
        elif not isq[i] and bit_of(i) == 0:
            acc += w[i]


def _split(order, node_of, bit_of):
    """Stable split of every node (run of equal node_of) by bit_of."""
    new, k = [], 0
    while k < len(order):
        j = k
        while j < len(order) and node_of(order[j]) == node_of(order[k]):
            j += 1
        run = order[k:j]
        new += [i for i in run if bit_of(i) == 0] + [i for i in run if bit_of(i) == 1]
        k = j
    return new


def _pipeline(D, Q, w, gS, cap, ns0=False, ns1=False, pair_max=0):
    nD = D.shape[0]
    P = np.concatenate([D, Q])
    n = P.shape[0]
    isq = np.arange(n) >= nD
    r0, r1 = _ranks(P[:, 0], nD, ns0), _ranks(P[:, 1], nD, ns1)
    b0, b1 = _bits(r0), _bits(r1)
    gS = min(gS, b0)
    wf = np.concatenate([w, np.zeros(len(Q), np.int64)])
    out = np.zeros(n, np.int64)
    xo = list(np.lexsort((~isq, P[:, 2])))  # last coordinate, queries first on ties
    groups = {}
    for i in xo:
        groups.setdefault(r0[i] >> gS, []).append(i)
    big = {g for g, pts in groups.items() if len(pts) > cap} if gS else set()

    def hbm_level(lv, pts):  # the records of level lv of the points pts, through "HBM"
        recs = []
        for i in pts:
            if ((r0[i] >> lv) & 1) != int(isq[i]):
                continue
            for j in range(b1):
                if ((r1[i] >> j) & 1) == int(isq[i]):
                    recs.append((i, j))
        recs.sort(key=lambda t: (r0[t[0]] >> (lv + 1), t[1], r1[t[0]] >> (t[1] + 1)))  # stable
        acc, prev = 0, None
        for i, j in recs:
            key = (r0[i] >> (lv + 1), j, r1[i] >> (j + 1))
            if key != prev:
                acc, prev = 0, key
            if isq[i]:
                out[i] += acc
            else:
                acc += wf[i]

    low_hbm = [i for i in xo if (r0[i] >> gS) in big]
    for lv in range(b0):
        hbm_level(lv, xo if lv >= gS else low_hbm)
    for g, pts in groups.items():
        if gS == 0 or g in big:
            continue
        # dense ranks of the second rank among the group's points
        u = sorted(set(int(r1[i]) for i in pts))
        loc = {i: u.index(int(r1[i])) for i in pts}
        nb1 = _bits(np.array([len(u) - 1]))
        order = list(pts)  # the order of level gS-1: the last coordinate
        for lv in range(gS - 1, -1, -1):
            blk = {i: r0[i] >> (lv + 1) for i in order}
            sizes = {}
            for i in order:
                sizes[blk[i]] = sizes.get(blk[i], 0) + 1
            if max(sizes.values()) <= pair_max:
                for p, i in enumerate(order):  # by pairs, within the block
                    if isq[i] and (r0[i] >> lv) & 1:
                        for k in range(p - 1, -1, -1):
                            d = order[k]
                            if blk[d] != blk[i]:
                                break
                            if not isq[d] and not (r0[d] >> lv) & 1 and loc[d] < loc[i]:
                                out[i] += wf[d]
                order = _split(order, lambda i, lv=lv: r0[i] >> (lv + 1), lambda i, lv=lv: (r0[i] >> lv) & 1)
                continue
            inner = [i for i in order if ((r0[i] >> lv) & 1) == int(isq[i])]
            for j in range(nb1 - 1, -1, -1):
                node = lambda i, j=j: (blk[i], loc[i] >> (j + 1))
                bit = lambda i, j=j: (loc[i] >> j) & 1
                _scan(inner, node, bit, isq, wf, out)
                inner = _split(inner, node, bit)
            order = _split(order, lambda i, lv=lv: r0[i] >> (lv + 1), lambda i, lv=lv: (r0[i] >> lv) & 1)
    return out[nD:]


def _brute(D, Q, w, ns0=False, ns1=False):
    c0 = (D[None, :, 0] <= Q[:, None, 0]) if ns0 else (D[None, :, 0] < Q[:, None, 0])
    c1 = (D[None, :, 1] <= Q[:, None, 1]) if ns1 else (D[None, :, 1] < Q[:, None, 1])
    dom = c0 & c1 & (D[None, :, 2] < Q[:, None, 2])
    return (dom * w[None, :]).sum(axis=1)


@pytest.mark.parametrize("ns0,ns1", [(False, False), (True, False), (False, True), (True, True)])
def test_group3_levels_equal_definition(ns0, ns1):
    rng = np.random.default_rng(2306 + 2 * ns0 + ns1)
    for _ in range(12):
        nD, nQ = int(rng.integers(0, 40)), int(rng.integers(1, 40))
        levels = int(rng.integers(1, 24))
        D = rng.integers(0, levels, size=(nD, 3))
        Q = rng.integers(0, levels, size=(nQ, 3))
        w = rng.integers(-9, 10, size=nD).astype(np.int64)
        want = _brute(D, Q, w, ns0, ns1)
        for gS in range(0, 7):
            for cap, pair_max in ((1000, 0), (8, 0), (1000, 6), (1000, 1000)):
                got = _pipeline(D, Q, w, gS, cap, ns0, ns1, pair_max)
                assert np.array_equal(got, want), (gS, cap, pair_max, nD, nQ, levels)


def test_group3_hand_case():
    """Four points per role; at gS = 2 one group holds every rank, so both
    first-rank levels run as blocks with local second ranks."""
    D = np.array([[0, 0, 0], [1, 2, 1], [2, 1, 2], [0, 3, 0]])
    Q = np.array([[3, 3, 3], [1, 3, 2], [2, 2, 3], [3, 1, 1]])
    w = np.array([1, 10, 100, 1000], np.int64)
    want = _brute(D, Q, w)
    assert want.tolist() == [111, 1, 1, 1]
    for gS in (0, 1, 2):
        for cap in (1000, 3):
            assert _pipeline(D, Q, w, gS, cap).tolist() == want.tolist()
