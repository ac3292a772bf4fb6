"""Pins of the CPU oracle to things other than itself (runs without a GPU).

Each test ties the oracle to the paper's worked examples, to its lemmas, to
textbook routines, to closed forms or to brute force on tiny inputs.  The
planted-mistake tests at the end build deliberately wrong oracles and check
that these pins catch them.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2305_16751_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


# --- worked examples printed in the paper -------------------------------

def test_sscan_worked_example():
    lines = dict(ln.split(":", 1) for ln in _golden_lines("sscan_example.txt"))
    a = [int(x) for x in lines["a"].split()]
    t = [int(x) for x in lines["t"].split()]
    want = [int(x) for x in lines["out"].split()]
    assert oracle.sscan_i64(a, t).tolist() == want


def test_prefix_set_worked_example():
    for ln in _golden_lines("prefix_sets.txt"):
        left, right = ln.split(":")
        x, b, which = left.split()
        want = sorted("" if s == "-" else s for s in right.split())
        got = sorted(oracle.prefix_set(int(x, 2), int(b), int(which)))
        assert got == want, ln


def _hand_case():
    D, w, Q, want_sum, want_cnt = [], [], [], [], []
    for ln in _golden_lines("hand_case_m2.txt"):
        f = ln.split()
        if f[0] == "D":
            D.append([int(f[1]), int(f[2])])
            w.append(int(f[3]))
        else:
            Q.append([int(f[1]), int(f[2])])
            want_sum.append(int(f[3]))
            want_cnt.append(int(f[4]))
    return (np.array(D, np.int32), np.array(Q, np.int32), np.array(w, np.int64),
            want_sum, want_cnt)


def test_hand_case_brute_and_sortscan():
    D, Q, w, want_sum, want_cnt = _hand_case()
    assert oracle.brute(D, Q, w, "sum")[0].tolist() == want_sum
    assert oracle.sortscan(D, Q, w, "sum")[0].tolist() == want_sum
    assert oracle.brute(D, Q, None, "count")[0].tolist() == want_cnt
    assert oracle.sortscan(D, Q, None, "count")[0].tolist() == want_cnt
    # max: w = 5, 7, 1 -> max over the dominated sets
    want_max = [5, 7, 7, np.iinfo(np.int32).min]
    assert oracle.brute(D, Q, w.astype(np.int32), "max")[0].tolist() == want_max
    assert oracle.sortscan(D, Q, w.astype(np.int32), "max")[0].tolist() == want_max


# --- Lemma 1 and Lemma 2 (Sec. 3) ---------------------------------------

@pytest.mark.parametrize("b", range(1, 8))
def test_lemma1_exhaustive(b):
    """x < y iff P0(x) and P1(y) share exactly one element, else none."""
    P0 = [set(oracle.prefix_set(x, b, 0)) for x in range(2**b)]
    P1 = [set(oracle.prefix_set(y, b, 1)) for y in range(2**b)]
    for x in range(2**b):
        for y in range(2**b):
            inter = P0[x] & P1[y]
            assert len(inter) == (1 if x < y else 0), (x, y, inter)


def test_lemma2_random_tuples():
    rng = np.random.default_rng(12)
    for _ in range(400):
        m = int(rng.integers(2, 4))
        b = [int(rng.integers(1, 7)) for _ in range(m)]
        x = [int(rng.integers(0, 2**bi)) for bi in b]
        y = [int(rng.integers(0, 2**bi)) for bi in b]
        P0 = set(itertools.product(*[oracle.prefix_set(x[i], b[i], 0) for i in range(m)]))
        P1 = set(itertools.product(*[oracle.prefix_set(y[i], b[i], 1) for i in range(m)]))
        dom = all(x[i] < y[i] for i in range(m))
        assert len(P0 & P1) == (1 if dom else 0)


# --- m = 1 is prefix aggregation (Sec. 1.1): a textbook routine ---------

@pytest.mark.parametrize("dtype", ["i32", "f32"])
def test_m1_is_prefix_sum(dtype):
    rng = np.random.default_rng(5)
    for _ in range(30):
        nD, nQ = int(rng.integers(0, 200)), int(rng.integers(0, 200))
        D, Q, w = workloads.random_small(rng, 1, nD, nQ, 9, dtype, "i64")
        order = np.argsort(D[:, 0], kind="stable")
        keys = D[order, 0]
        csum = np.concatenate([[0], np.cumsum(w[order])])
        want = csum[np.searchsorted(keys, Q[:, 0], side="left")]
        assert oracle.brute(D, Q, w, "sum")[0].tolist() == want.tolist()
        assert oracle.sortscan(D, Q, w, "sum")[0].tolist() == want.tolist()


# --- the two oracles agree on tiny tied inputs --------------------------

CASES = [(m, dt, wt, op) for m in (1, 2, 3, 4) for dt in ("i32", "f32")
         for wt, op in (("i64", "sum"), ("f32", "sum"), ("i32", "max"), ("f32", "max"), ("i64", "count"),
                        ("i32", "min"), ("f32", "min"))]


@pytest.mark.parametrize("m,dt,wt,op", CASES)
def test_brute_equals_sortscan(m, dt, wt, op):
    rng = np.random.default_rng(1000 + m)
    for _ in range(12):
        nD, nQ = int(rng.integers(0, 40)), int(rng.integers(0, 40))
        levels = int(rng.integers(1, 7))
        D, Q, w = workloads.random_small(rng, m, nD, nQ, levels, dt, wt)
        a, S = oracle.brute(D, Q, w, op)
        b, _ = oracle.sortscan(D, Q, w, op)
        if wt == "f32" and op == "sum":
            assert np.allclose(a, b, rtol=0, atol=1e-12 * (1 + S.max(initial=0)))
        else:
            assert a.tolist() == b.tolist()


def test_brute_equals_sortscan_medium():
    rng = np.random.default_rng(77)
    for m in (2, 3):
        D, Q, w = workloads.random_small(rng, m, 600, 500, 50, "i32", "i64")
        assert oracle.brute(D, Q, w, "sum")[0].tolist() == oracle.sortscan(D, Q, w, "sum")[0].tolist()


def _brute_py(D, Q, w, op):
    """Pure-Python definition for tiny inputs (independent of the C code).
    Integer weights give Python ints; float weights give Python floats (the
    sum in double, max / min exact, +-inf for the empty set)."""
    is_float = w is not None and np.asarray(w).dtype.kind == "f"
    out = []
    for q in Q:
        dom = [i for i, d in enumerate(D) if all(d[k] < q[k] for k in range(len(q)))]
        if op == "count":
            out.append(len(dom))
        elif is_float:
            vals = [float(w[i]) for i in dom]
            if op == "sum":
                out.append(float(sum(vals)))
            elif op == "min":
                out.append(min(vals, default=float("inf")))
            else:
                out.append(max(vals, default=float("-inf")))
        elif op == "sum":
            out.append(int(sum(int(w[i]) for i in dom)))
        elif op == "min":
            out.append(min([int(w[i]) for i in dom], default=np.iinfo(np.int32).max))
        else:
            out.append(max([int(w[i]) for i in dom], default=np.iinfo(np.int32).min))
    return out


def test_brute_equals_python_definition():
    rng = np.random.default_rng(3)
    for _ in range(40):
        m = int(rng.integers(1, 4))
        D, Q, w = workloads.random_small(rng, m, 25, 20, 5, "i32", "i32")
        for op in ("sum", "max", "count", "min"):
            assert oracle.brute(D, Q, w, op)[0].tolist() == _brute_py(D, Q, w, op)


def test_brute_float_weights_equal_python_definition():
    """The float branch of F (max, min and the double sum of float32
    weights) against the pure-Python definition: the C oracle's brute force
    and its sort-and-scan share that branch, so this pins it independently."""
    rng = np.random.default_rng(4)
    for _ in range(40):
        m = int(rng.integers(1, 4))
        D, Q, w = workloads.random_small(rng, m, 25, 20, 5, "f32", "f32")
        for op in ("max", "min"):
            assert oracle.brute(D, Q, w, op)[0].tolist() == _brute_py(D, Q, w, op)
        got = oracle.brute(D, Q, w, "sum")[0]
        want = np.array(_brute_py(D, Q, w, "sum"))
        assert np.allclose(got, want, rtol=0, atol=1e-12 * (1 + np.abs(w).sum()))


def test_min_is_negated_max_of_negated_weights():
    """min F = -max(-w) (an identity the MIN code does not use), and the
    empty set gives +inf / INT32_MAX."""
    rng = np.random.default_rng(31)
    for m in (1, 2, 3):
        D, Q, w = workloads.random_small(rng, m, 300, 200, 9, "i32", "i32")
        w = np.maximum(w, np.iinfo(np.int32).min + 1)
        mn = oracle.sortscan(D, Q, w, "min")[0]
        mx = oracle.sortscan(D, Q, -w, "max")[0]
        empty = mx == np.iinfo(np.int32).min
        assert np.array_equal(mn[~empty], -mx[~empty])
        assert np.all(mn[empty] == np.iinfo(np.int32).max)
        wf = rng.standard_normal(300).astype(np.float32)
        mnf = oracle.brute(D, Q, wf, "min")[0]
        mxf = oracle.brute(D, Q, -wf, "max")[0]
        assert np.array_equal(np.isposinf(mnf), np.isneginf(mxf))
        fin = np.isfinite(mnf)
        assert np.array_equal(mnf[fin], -mxf[fin])


# --- record count law (Sec. 5 flat map) ----------------------------------

def _record_count_formula(D, Q):
    """T = sum over data of prod_i zeros(r_i) + sum over queries of
    prod_i ones(r_i), ranks dense 0-based with b_i = ceil(log2 U_i) digits."""
    m = D.shape[1]
    P = np.concatenate([D, Q]).astype(np.float64)
    nD = D.shape[0]
    cnt = np.ones(P.shape[0], dtype=np.int64)
    bmax = 0
    for i in range(m - 1):
        u = np.unique(P[:, i])
        r = np.searchsorted(u, P[:, i])
        b = int(np.ceil(np.log2(len(u)))) if len(u) > 1 else 0
        bmax = max(bmax, b)
        ones = np.array([bin(int(v)).count("1") for v in r], dtype=np.int64)
        cnt *= np.where(np.arange(P.shape[0]) < nD, b - ones, ones)
    return int(cnt.sum()), bmax


def test_record_count_law():
    rng = np.random.default_rng(8)
    for m in (1, 2, 3):
        for _ in range(10):
            D, Q, _ = workloads.random_small(rng, m, 150, 130, int(rng.integers(2, 300)), "i32", "i64")
            T = oracle.record_count(D, Q)
            want, b = _record_count_formula(D, Q)
            assert T == want
            assert T <= (D.shape[0] + Q.shape[0]) * max(b, 1) ** (m - 1)


# --- edge cases the method has ------------------------------------------

def test_empty_inputs():
    D = np.zeros((0, 2), np.int32)
    Q = np.array([[1, 1], [5, 5]], np.int32)
    assert oracle.brute(D, Q, np.zeros(0, np.int64), "sum")[0].tolist() == [0, 0]
    assert oracle.sortscan(D, Q, np.zeros(0, np.int64), "sum")[0].tolist() == [0, 0]
    assert oracle.sortscan(D, Q, np.zeros(0, np.int32), "max")[0].tolist() == [np.iinfo(np.int32).min] * 2
    out, _ = oracle.sortscan(Q, np.zeros((0, 2), np.int32), np.ones(2, np.int64), "sum")
    assert out.shape == (0,)


def test_all_points_equal_give_unit():
    D = np.full((50, 3), 7, np.int32)
    Q = np.full((40, 3), 7, np.int32)
    out, T = oracle.sortscan(D, Q, np.ones(50, np.int64), "sum")
    assert out.tolist() == [0] * 40 and T == 0
    out, _ = oracle.sortscan(D, Q, np.ones(50, np.float32), "max")
    assert np.all(np.isneginf(out))


def test_signed_zero_is_one_coordinate():
    D = np.array([[-0.0, 1.0]], np.float32)
    Q = np.array([[0.0, 2.0], [0.5, 2.0]], np.float32)
    for f in (oracle.brute, oracle.sortscan):
        assert f(D, Q, np.array([3], np.int64), "sum")[0].tolist() == [0, 3]


def test_infinities_are_ordered():
    D = np.array([[-np.inf, -np.inf], [1.0, np.inf]], np.float32)
    Q = np.array([[0.0, 0.0], [np.inf, np.inf], [2.0, 5.0]], np.float32)
    w = np.array([1, 10], np.int64)
    for f in (oracle.brute, oracle.sortscan):
        assert f(D, Q, w, "sum")[0].tolist() == [1, 1, 1]


def test_nan_coordinate_is_an_error():
    D = np.array([[np.nan, 1.0]], np.float32)
    Q = np.array([[1.0, 1.0]], np.float32)
    for f in (oracle.brute, oracle.sortscan):
        with pytest.raises(oracle.OracleError) as e:
            f(D, Q, np.ones(1, np.int64), "sum")
        assert e.value.code == 6


def test_strictness_in_every_coordinate():
    # ties in one coordinate exclude the point, whatever the other ones say
    D = np.array([[1, 1], [1, 0], [0, 1], [0, 0]], np.int32)
    Q = np.array([[1, 1]], np.int32)
    w = np.array([1, 10, 100, 1000], np.int64)
    for f in (oracle.brute, oracle.sortscan):
        assert f(D, Q, w, "sum")[0].tolist() == [1000]


def test_int64_sum_wraps():
    D = np.array([[0, 0], [1, 1]], np.int32)
    Q = np.array([[5, 5]], np.int32)
    w = np.array([2**62, 2**62], np.int64)
    for f in (oracle.brute, oracle.sortscan):
        assert f(D, Q, w * 2, "sum")[0].tolist() == [0]  # 2^64 wraps to 0


# --- backward: transposed sum vs central finite differences -------------

def test_backward_transpose_vs_finite_differences():
    rng = np.random.default_rng(2305)
    n = 512
    D = workloads.grid24(rng, (n, 2))
    Q = workloads.grid24(rng, (n, 2))
    # weights and step on a 2^-10 grid so w +- h is exact in float32
    w = (rng.integers(-2048, 2048, size=n) * 2.0**-10).astype(np.float32)
    c = rng.standard_normal(n).astype(np.float32)
    grad, _ = oracle.brute_transpose(D, Q, c)
    h = 2.0**-10

    def L(wv):
        out, _ = oracle.brute(D, Q, wv, "sum")
        return float(np.dot(c.astype(np.float64), out))

    fd = np.empty(n)
    for d in range(n):
        wp, wm = w.copy(), w.copy()
        wp[d] += np.float32(h)
        wm[d] -= np.float32(h)
        fd[d] = (L(wp) - L(wm)) / (2 * h)
    assert np.allclose(fd, grad, rtol=1e-9, atol=1e-9)


def test_backward_transpose_is_reverse_dominance():
    rng = np.random.default_rng(9)
    D, Q, _ = workloads.random_small(rng, 3, 60, 70, 5, "i32", "i64")
    g = rng.standard_normal(70).astype(np.float32)
    grad, _ = oracle.brute_transpose(D, Q, g)
    # reverse dominance with negated coordinates is the forward problem
    fwd, _ = oracle.brute(-Q, -D, g, "sum")
    assert np.allclose(grad, fwd, rtol=0, atol=1e-12)


# --- planted mistakes are caught by the pins ----------------------------

def _pins_pass(plant):
    D, Q, w, want_sum, _ = _hand_case()
    if oracle.brute(D, Q, w, "sum", plant=plant)[0].tolist() != want_sum:
        return False
    if oracle.sortscan(D, Q, w, "sum", plant=plant)[0].tolist() != want_sum:
        return False
    rng = np.random.default_rng(44)
    for m in (1, 2, 3):
        for _ in range(10):
            D, Q, w = workloads.random_small(rng, m, 30, 30, 4, "i32", "i64")
            if oracle.brute(D, Q, w, "sum", plant=plant)[0].tolist() != _brute_py(D, Q, w, "sum"):
                return False
            if oracle.sortscan(D, Q, w, "sum", plant=plant)[0].tolist() != _brute_py(D, Q, w, "sum"):
                return False
    return True


def test_real_oracle_passes_the_pins():
    assert _pins_pass(0)


@pytest.mark.parametrize("plant", [1, 2, 3, 4])
def test_planted_mistakes_are_caught(plant):
    # 1: non-strict dominance; 2: data before queries on a tie of the last
    # coordinate; 3: one binary digit too few per rank; 4: the last coordinate
    # also splits segments
    assert not _pins_pass(plant)


# --- non-strict coordinates (an extension of the strict order) -----------

def _brute_py_ns(D, Q, w, nonstrict):
    out = []
    for q in Q:
        tot = 0
        for i, d in enumerate(D):
            if all((d[k] <= q[k]) if (nonstrict >> k) & 1 else (d[k] < q[k]) for k in range(len(q))):
                tot += int(w[i])
        out.append(tot)
    return out


def test_nonstrict_brute_equals_python_definition():
    rng = np.random.default_rng(41)
    for _ in range(30):
        m = int(rng.integers(1, 4))
        D, Q, w = workloads.random_small(rng, m, 25, 20, 4, "i32", "i64")
        mask = int(rng.integers(0, 1 << m))
        assert oracle.brute(D, Q, w, "sum", nonstrict=mask)[0].tolist() == _brute_py_ns(D, Q, w, mask)


def test_nonstrict_on_integers_is_strict_against_the_successor():
    """For integer coordinates d <= q  <=>  d < q + 1: shifting the queries'
    non-strict coordinates by one turns the strict oracle into the
    non-strict one."""
    rng = np.random.default_rng(42)
    for m in (1, 2, 3):
        for mask in range(1, 1 << m):
            D, Q, w = workloads.random_small(rng, m, 400, 300, 6, "i32", "i64")
            Q1 = Q.copy()
            for k in range(m):
                if (mask >> k) & 1:
                    Q1[:, k] += 1
            a = oracle.brute(D, Q, w, "sum", nonstrict=mask)[0]
            b = oracle.sortscan(D, Q1, w, "sum")[0]
            assert a.tolist() == b.tolist()


def test_nonstrict_without_ties_equals_strict():
    rng = np.random.default_rng(43)
    P = rng.permutation(2000).reshape(1000, 2).astype(np.int32)
    D, Q = P[:600], P[600:]
    w = rng.integers(-9, 10, 600).astype(np.int64)
    for mask in range(4):
        assert oracle.brute(D, Q, w, "sum", nonstrict=mask)[0].tolist() == oracle.brute(D, Q, w, "sum")[0].tolist()


# --- the O(n log n) sweep for m = 2 (full-size checks) -------------------

SWEEP_CASES = [(dt, wt, op) for dt in ("i32", "f32")
               for wt, op in (("i64", "sum"), ("f32", "sum"), ("i32", "max"), ("f32", "max"), ("i64", "count"),
                              ("i32", "min"), ("f32", "min"))]


@pytest.mark.parametrize("dt,wt,op", SWEEP_CASES)
def test_sweep2_equals_brute(dt, wt, op):
    """The Fenwick-tree sweep (not the paper's algorithm) equals the
    definition on tied inputs, for every op and comparison mask."""
    rng = np.random.default_rng(2000 + len(dt) + len(op))
    for _ in range(10):
        nD, nQ = int(rng.integers(0, 300)), int(rng.integers(0, 300))
        D, Q, w = workloads.random_small(rng, 2, nD, nQ, int(rng.integers(1, 12)), dt, wt)
        for mask in range(4):
            a, Sa = oracle.brute(D, Q, w, op, nonstrict=mask)
            b, Sb = oracle.sweep2(D, Q, w, op, nonstrict=mask)
            assert np.allclose(Sa, Sb, rtol=1e-12, atol=0)
            if wt == "f32" and op == "sum":
                assert np.allclose(a, b, rtol=0, atol=1e-12 * (1 + Sa.max(initial=0)))
            else:
                assert a.tolist() == b.tolist()


def test_sweep2_python_definition_and_hand_case():
    D, Q, w, want_sum, want_cnt = _hand_case()
    assert oracle.sweep2(D, Q, w, "sum")[0].tolist() == want_sum
    assert oracle.sweep2(D, Q, None, "count")[0].tolist() == want_cnt
    rng = np.random.default_rng(6)
    for _ in range(30):
        D, Q, w = workloads.random_small(rng, 2, 30, 25, 4, "i32", "i32")
        for op in ("sum", "max", "min", "count"):
            assert oracle.sweep2(D, Q, w, op)[0].tolist() == _brute_py(D, Q, w, op)


def test_sweep2_transpose_equals_brute():
    rng = np.random.default_rng(7)
    for _ in range(12):
        D, Q, _ = workloads.random_small(rng, 2, int(rng.integers(0, 200)), int(rng.integers(0, 200)), 6,
                                         "f32", "i64")
        g = rng.standard_normal(Q.shape[0]).astype(np.float32)
        grad, S = oracle.sweep2_transpose(D, Q, g)
        want, Sw = oracle.brute_transpose(D, Q, g)
        assert np.allclose(grad, want, rtol=0, atol=1e-12 * (1 + Sw.max(initial=0)))
        assert np.allclose(S, Sw, rtol=1e-12, atol=0)
        for mask in range(1, 4):
            # d_i <= q_i  <=>  -q_i <= -d_i: the non-strict adjoint is the
            # non-strict forward problem with negated coordinates, roles swapped
            gm, _ = oracle.sweep2_transpose(D, Q, g, nonstrict=mask)
            fm, Sm = oracle.brute(-Q, -D, g, "sum", nonstrict=mask)
            assert np.allclose(gm, fm, rtol=0, atol=1e-12 * (1 + Sm.max(initial=0)))


def test_sweep2_edge_cases():
    D = np.zeros((0, 2), np.float32)
    Q = np.array([[1, 1], [5, 5]], np.float32)
    assert oracle.sweep2(D, Q, np.zeros(0, np.int32), "max")[0].tolist() == [np.iinfo(np.int32).min] * 2
    assert oracle.sweep2(Q, D, np.ones(2, np.int64), "sum")[0].shape == (0,)
    E = np.full((20, 2), 3.0, np.float32)
    assert oracle.sweep2(E, E, np.ones(20, np.int64), "sum")[0].tolist() == [0] * 20
    assert oracle.sweep2(E, E, np.ones(20, np.int64), "sum", nonstrict=3)[0].tolist() == [20] * 20
    Z = np.array([[-0.0, 1.0]], np.float32)
    assert oracle.sweep2(Z, np.array([[0.0, 2.0], [0.5, 2.0]], np.float32), np.array([3], np.int64),
                         "sum")[0].tolist() == [0, 3]
    with pytest.raises(oracle.OracleError):
        oracle.sweep2(np.array([[np.nan, 1.0]], np.float32), Q, np.ones(1, np.int64), "sum")


def _sweep_pins_pass(plant):
    D, Q, w, want_sum, _ = _hand_case()
    if oracle.sweep2(D, Q, w, "sum", plant=plant)[0].tolist() != want_sum:
        return False
    rng = np.random.default_rng(45)
    for _ in range(20):
        D, Q, w = workloads.random_small(rng, 2, 40, 40, 4, "i32", "i64")
        if oracle.sweep2(D, Q, w, "sum", plant=plant)[0].tolist() != _brute_py(D, Q, w, "sum"):
            return False
    return True


def test_real_sweep_passes_the_pins():
    assert _sweep_pins_pass(0)


@pytest.mark.parametrize("plant", [5, 6])
def test_planted_sweep_mistakes_are_caught(plant):
    # 5: data before queries on a tie of the last coordinate; 6: the query's
    # own first-coordinate rank included (non-strict)
    assert not _sweep_pins_pass(plant)
