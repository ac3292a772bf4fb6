"""The level-wise formulation's mathematics, on the CPU (no GPU, no CUDA
code): a plain Python model of the passes -- points in the order of the last
coordinate (queries first on ties, Sec. 5), two rank levels per pass from the
top, a segmented scan of three binary-trie channels inside each prefix group,
then a stable partition of the whole array by the 2-bit digit -- equals the
definition of the dominance sum (brute force) on small random inputs with
heavy ties, for odd and even rank bit counts.  This pins the reading the
GPU variant "wavelet" implements: at the highest rank bit where d and q
differ, d has 0 and q has 1 (Lemma 1), so within a pass a query receives F
over the preceding data of its group with a smaller digit."""
import numpy as np


def _dense_ranks(x):
    _, r = np.unique(x, return_inverse=True)
    return r.astype(np.int64)


def _levelwise(D, Q, w, F=np.add, e=0):
    nD, nQ = D.shape[0], Q.shape[0]
    P = np.concatenate([D, Q])
    isq = np.arange(nD + nQ) >= nD
    r = _dense_ranks(P[:, 0])
    b = max(1, int(np.ceil(np.log2(r.max() + 1))) if r.max() > 0 else 1)
    # order of the last coordinate, queries first on ties
    order = np.lexsort((~isq, P[:, -1]))
    key, q, idx = r[order], isq[order], order
    val = np.where(q, e, np.concatenate([w, np.zeros(nQ, w.dtype)])[order]).astype(np.int64)
    acc = np.full(len(order), e, np.int64)
    top = b
    while top > 0:
        width = 2 if top >= 2 else 1
        s = top - width
        grp, dig = key >> (s + width), (key >> s) & ((1 << width) - 1)
        nch = (1 << width) - 1
        run = np.full(nch, e, np.int64)
        for i in range(len(key)):
            if i == 0 or grp[i] != grp[i - 1]:
                run[:] = e
            for t in range(width - 1, -1, -1):
                ch = ((1 << width) + int(dig[i])) >> (t + 1)  # trie node (heap numbering) at digit bit t
                bit = (int(dig[i]) >> t) & 1
                if q[i] and bit == 1:
                    acc[i] = F(acc[i], run[ch - 1])
                if not q[i] and bit == 0:
                    run[ch - 1] = F(run[ch - 1], val[i])
        perm = np.argsort(dig, kind="stable")
        key, q, val, acc, idx = key[perm], q[perm], val[perm], acc[perm], idx[perm]
        top -= width
    out = np.full(nD + nQ, e, np.int64)
    out[idx] = acc
    return out[nD:]


def _levelwise_sum(D, Q, w):
    return _levelwise(D, Q, w)


def _brute(D, Q, w):
    less = np.all(D[None, :, :] < Q[:, None, :], axis=2)
    return (less * w[None, :]).sum(axis=1)


def _brute_max(D, Q, w, e):
    less = np.all(D[None, :, :] < Q[:, None, :], axis=2)
    return np.where(less, w[None, :], e).max(axis=1, initial=e)


def test_levelwise_model_equals_definition():
    rng = np.random.default_rng(2305)
    for trial in range(120):
        nD, nQ = int(rng.integers(0, 40)), int(rng.integers(1, 40))
        levels = int(rng.integers(1, 70))
        m = int(rng.integers(1, 3))
        D = rng.integers(0, levels, size=(nD, m))
        Q = rng.integers(0, levels, size=(nQ, m))
        w = rng.integers(-9, 10, size=nD)
        if m == 1:
            # the rank is the role bit: every datum below every query; the
            # comparison is the last coordinate alone
            D2 = np.concatenate([np.zeros((nD, 1), np.int64), D], axis=1)
            Q2 = np.concatenate([np.ones((nQ, 1), np.int64), Q], axis=1)
            got = _levelwise_sum(D2, Q2, w)
        else:
            got = _levelwise_sum(D, Q, w)
        assert np.array_equal(got, _brute(D, Q, w)), trial


def test_levelwise_model_single_pass_cases():
    # b = 1 (two ranks) and b = 2 (one full 2-bit pass): hand-checkable
    D = np.array([[0, 0], [1, 0], [0, 2]])
    Q = np.array([[1, 1], [1, 3], [0, 5]])
    w = np.array([5, 7, 11])
    assert np.array_equal(_levelwise_sum(D, Q, w), [5, 5 + 11, 0])
    D = np.array([[0, 0], [1, 1], [2, 2], [3, 3]])
    Q = np.array([[4, 4], [3, 9], [1, 1]])
    w = np.array([1, 10, 100, 1000])
    assert np.array_equal(_levelwise_sum(D, Q, w), [1111, 111, 1])


def test_levelwise_model_max():
    """The same passes with F = max (unit: the smallest int64) equal the
    definition: only associativity, commutativity and the unit are used."""
    rng = np.random.default_rng(2306)
    e = np.iinfo(np.int64).min
    for trial in range(80):
        nD, nQ = int(rng.integers(0, 30)), int(rng.integers(1, 30))
        levels = int(rng.integers(1, 50))
        D = rng.integers(0, levels, size=(nD, 2))
        Q = rng.integers(0, levels, size=(nQ, 2))
        w = rng.integers(-99, 100, size=nD)
        got = _levelwise(D, Q, w, F=np.maximum, e=e)
        assert np.array_equal(got, _brute_max(D, Q, w, e)), trial
