"""Non-strict coordinates, the basic (unimproved) variant of Sec. 4, and
dominance counting with D = Q (ECDF), on the GPU against the oracle."""
import numpy as np
import pytest

import oracle
from gpu_helpers import assert_matches_oracle, to_dev, torch
from paper_2305_16751_gb300 import domagg, workloads

pytestmark = pytest.mark.gpu


def _forward(D, Q, w, op, nonstrict=0, variant="improved"):
    out = domagg.forward(to_dev(D), to_dev(Q), to_dev(w), op, nonstrict=nonstrict, variant=variant)
    torch().cuda.synchronize()
    return out.cpu().numpy()


def _check(got, D, Q, w, op, nonstrict):
    want, S = oracle.brute(D, Q, w, op, nonstrict=nonstrict)
    assert_matches_oracle(got, D, Q, w, op, want=want, S=S)


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("dt,wt,op", [("i32", "i64", "sum"), ("f32", "f32", "sum"), ("i32", "i32", "max"),
                                      ("f32", "i64", "count")])
def test_nonstrict_masks_match_oracle(m, dt, wt, op):
    rng = np.random.default_rng(500 + 10 * m + len(op))
    for mask in range(1 << m):
        D, Q, w = workloads.random_small(rng, m, 5000, 4000, 30, dt, wt)
        wv = None if op == "count" else w
        _check(_forward(D, Q, wv, op, nonstrict=mask), D, Q, wv, op, mask)


def test_all_equal_points_nonstrict_dominate_everything():
    D = np.full((3000, 2), 5, np.int32)
    Q = np.full((1000, 2), 5, np.int32)
    w = np.arange(3000, dtype=np.int64)
    assert np.all(_forward(D, Q, w, "sum", nonstrict=3) == w.sum())
    assert np.all(_forward(D, Q, w, "sum", nonstrict=1) == 0)  # strict in the last coordinate


def _basic_record_count(D, Q):
    """Records of the basic variant: every coordinate a bitstring, so
    T = sum over data of prod_i zeros(r_i) + sum over queries of prod_i ones(r_i)."""
    P = np.concatenate([D, Q]).astype(np.float64)
    P[P == 0] = 0.0
    nD = D.shape[0]
    cnt = np.ones(P.shape[0], dtype=np.int64)
    for i in range(P.shape[1]):
        u, r = np.unique(P[:, i], return_inverse=True)
        b = int(np.ceil(np.log2(len(u)))) if len(u) > 1 else 0
        ones = np.zeros(P.shape[0], np.int64)
        for j in range(b):
            ones += (r >> j) & 1
        cnt *= np.where(np.arange(P.shape[0]) < nD, b - ones, ones)
    return int(cnt.sum())


@pytest.mark.parametrize("m", [1, 2])
@pytest.mark.parametrize("dt,wt,op", [("i32", "i64", "sum"), ("f32", "f32", "sum"), ("i32", "i32", "max")])
def test_basic_variant_equals_definition(m, dt, wt, op):
    rng = np.random.default_rng(600 + m)
    for nD, nQ, levels in ((4000, 3000, 25), (2500, 2500, 2000), (1, 5000, 3)):
        D, Q, w = workloads.random_small(rng, m, nD, nQ, levels, dt, wt)
        got = _forward(D, Q, w, op, variant="basic")
        _check(got, D, Q, w, op, 0)
        if op == "sum":
            assert domagg.stats()["n_records"] == _basic_record_count(D, Q)
            improved = _forward(D, Q, w, op)
            if wt == "i64":
                assert np.array_equal(got, improved)


def test_basic_variant_at_scale_m2():
    """|D| = |Q| = 2^18 uniform float32 points: the basic variant's n log^2 n
    records give the same sums as the Sec. 5 pipeline (sampled against the
    oracle); its record count is the basic flat-map formula."""
    rng = np.random.default_rng(7)
    n = 1 << 18
    D = (rng.integers(0, 1 << 24, size=(n, 2)) * 2.0**-24).astype(np.float32)
    Q = (rng.integers(0, 1 << 24, size=(n, 2)) * 2.0**-24).astype(np.float32)
    w = rng.integers(-1000, 1001, size=n).astype(np.int64)
    basic = _forward(D, Q, w, "sum", variant="basic")
    T_basic = domagg.stats()["n_records"]
    improved = _forward(D, Q, w, "sum")
    T_improved = domagg.stats()["n_records"]
    assert np.array_equal(basic, improved)
    assert T_basic == _basic_record_count(D, Q) and T_basic > 4 * T_improved
    qi = np.sort(rng.choice(n, 128, replace=False))
    assert_matches_oracle(basic, D, Q, w, "sum", qidx=qi)


def test_ecdf_counts_and_two_sample_statistic():
    """Dominance counting with D = Q and every coordinate non-strict is the
    empirical CDF at the sample points; the two-sample statistic
    max |F_X - F_Y| over X u Y matches the oracle's."""
    p = workloads.ecdf_samples(n=6000, m=3)
    X, Y = p.D, p.Q
    cnt = _forward(X, X, None, "count", nonstrict=7)
    want = oracle.brute(X, X, None, "count", nonstrict=7)[0]
    assert np.array_equal(cnt, want)
    ks = domagg.ks_statistic(to_dev(X), to_dev(Y))
    Z = np.concatenate([X, Y])
    fx = oracle.brute(X, Z, None, "count", nonstrict=7)[0] / X.shape[0]
    fy = oracle.brute(Y, Z, None, "count", nonstrict=7)[0] / Y.shape[0]
    assert abs(ks - np.abs(fx - fy).max()) < 1e-12


def test_ecdf_distance_entry_point():
    """domagg_ecdf_distance on given counts: the largest |cx/nx - cy/ny|
    (a hand case, then no points at all), and its argument checks."""
    t = torch()
    h = domagg.handle(0)
    cx = t.tensor([0, 3, 5, 10], dtype=t.int64, device="cuda")
    cy = t.tensor([1, 1, 4, 4], dtype=t.int64, device="cuda")
    out = t.full((1,), -1.0, dtype=t.float64, device="cuda")
    st = domagg.lib().domagg_ecdf_distance(h, domagg._ptr(cx), domagg._ptr(cy), 4, 10, 4, domagg._ptr(out), None)
    assert st == 0
    assert abs(out.item() - max(abs(a / 10 - b / 4) for a, b in zip([0, 3, 5, 10], [1, 1, 4, 4]))) < 1e-15
    st = domagg.lib().domagg_ecdf_distance(h, None, None, 0, 10, 4, domagg._ptr(out), None)
    assert st == 0 and out.item() == 0.0
    assert domagg.lib().domagg_ecdf_distance(h, domagg._ptr(cx), domagg._ptr(cy), 4, 0, 4, domagg._ptr(out), None) == 1
    assert domagg.lib().domagg_ecdf_distance(h, domagg._ptr(cx), None, 4, 10, 4, domagg._ptr(out), None) == 1


def test_variant_arguments_are_checked():
    D = np.zeros((4, 4), np.int32)
    with pytest.raises(domagg.DomaggError) as e:
        _forward(D, D, np.ones(4, np.int64), "sum", variant="basic")
    assert e.value.status == 2  # UNSUPPORTED: basic needs m <= 3
    with pytest.raises(domagg.DomaggError) as e:
        _forward(D[:, :2], D[:, :2], np.ones(4, np.int64), "sum", nonstrict=4)
    assert e.value.status == 1  # INVALID_ARG: mask bit beyond m


# --- m = 4 (the Sec. 5 pipeline with three rank coordinates) ---------------

@pytest.mark.parametrize("dt,wt,op", [("i32", "i64", "sum"), ("f32", "f32", "sum"), ("i32", "i32", "max"),
                                      ("f32", "i64", "count")])
def test_m4_matches_oracle(dt, wt, op):
    rng = np.random.default_rng(700 + len(op) + len(dt))
    for nD, nQ, levels in ((3000, 2500, 12), (1500, 1800, 300), (2, 4000, 4)):
        D, Q, w = workloads.random_small(rng, 4, nD, nQ, levels, dt, wt)
        wv = None if op == "count" else w
        _check(_forward(D, Q, wv, op), D, Q, wv, op, 0)
        if op == "sum" and dt == "i32":
            assert domagg.stats()["n_records"] == oracle.record_count(D, Q)


def test_m4_nonstrict_and_basic_m3():
    rng = np.random.default_rng(710)
    for mask in (1, 6, 8, 15):
        D, Q, w = workloads.random_small(rng, 4, 2000, 2000, 10, "i32", "i64")
        _check(_forward(D, Q, w, "sum", nonstrict=mask), D, Q, w, "sum", mask)
    D, Q, w = workloads.random_small(rng, 3, 2500, 2000, 40, "i32", "i64")
    got = _forward(D, Q, w, "sum", variant="basic")
    _check(got, D, Q, w, "sum", 0)
    assert domagg.stats()["n_records"] == _basic_record_count(D, Q)


def test_m4_in_a_batch_and_key_width_limit():
    rng = np.random.default_rng(720)
    probs = [workloads.random_small(rng, 1 + i % 4, 800 + 50 * i, 700, 30, "i32", "i64") for i in range(12)]
    outs = domagg.batch([(to_dev(D), to_dev(Q), to_dev(w)) for D, Q, w in probs], "sum")
    torch().cuda.synchronize()
    for (D, Q, w), o in zip(probs, outs):
        _check(o.cpu().numpy(), D, Q, w, "sum", 0)
    # 2^22 distinct values in every coordinate: b = 22, a 65-bit node key
    n = 1 << 21
    P = rng.permutation(np.arange(2 * n, dtype=np.int32))
    X = np.stack([P, np.roll(P, 1), np.roll(P, 2), np.roll(P, 3)], axis=1)
    with pytest.raises(domagg.DomaggError) as e:
        _forward(X[:n], X[n:], np.ones(n, np.int64), "sum")
    assert e.value.status == 2


@pytest.mark.parametrize("m", [1, 2, 3])
def test_nonstrict_backward_and_autograd(m):
    """The adjoint with non-strict coordinates: grad_w[d] = sum of g[q] over
    q with d <= q in the masked coordinates -- against the oracle run on the
    negated, role-swapped problem (d <= q  <=>  -q <= -d)."""
    rng = np.random.default_rng(800 + m)
    for mask in range(1, 1 << m):
        D, Q, _ = workloads.random_small(rng, m, 3000, 2500, 20, "i32", "f32")
        g = rng.standard_normal(2500).astype(np.float32)
        got = domagg.backward(to_dev(D), to_dev(Q), to_dev(g), nonstrict=mask).cpu().numpy()
        want, S = oracle.brute(-Q, -D, g, "sum", nonstrict=mask)
        assert_matches_oracle(got, -Q, -D, g, "sum", want=want, S=S)
    D, Q, w = workloads.random_small(rng, m, 2000, 1500, 15, "i32", "f32")
    c = rng.standard_normal(1500).astype(np.float32)
    wd = to_dev(w).requires_grad_(True)
    out = domagg.dominance_sum(to_dev(D), to_dev(Q), wd, (1 << m) - 1)
    (out * to_dev(c)).sum().backward()
    want, S = oracle.brute(-Q, -D, c, "sum", nonstrict=(1 << m) - 1)
    assert_matches_oracle(wd.grad.cpu().numpy(), -Q, -D, c, "sum", want=want, S=S)
