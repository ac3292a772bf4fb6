"""The level-wise formulation (variant "wavelet", m <= 2): the levels of the
first coordinate's rank evaluated on the points by segmented scans and
stable partitions, no flat-map records; on the GPU against the oracle."""
import numpy as np
import pytest

import oracle
from gpu_helpers import assert_matches_oracle, to_dev, torch
from paper_2305_16751_gb300 import domagg, workloads

pytestmark = pytest.mark.gpu


def _fw(D, Q, w, op, nonstrict=0, variant="wavelet"):
    out = domagg.forward(to_dev(D), to_dev(Q), None if w is None else to_dev(w), op, nonstrict=nonstrict,
                         variant=variant)
    torch().cuda.synchronize()
    return out.cpu().numpy()


def _check(D, Q, w, op, nonstrict=0):
    got = _fw(D, Q, w, op, nonstrict)
    want, S = oracle.brute(D, Q, w, op, nonstrict=nonstrict)
    assert_matches_oracle(got, D, Q, w, op, want=want, S=S)
    return got


CASES = [("i32", "i64", "sum"), ("f32", "f32", "sum"), ("i32", "i32", "max"), ("f32", "f32", "max"),
         ("i32", "i32", "min"), ("f32", "f32", "min"), ("f32", "i64", "count")]


@pytest.mark.parametrize("m", [1, 2])
@pytest.mark.parametrize("dt,wt,op", CASES)
def test_wavelet_matches_oracle(m, dt, wt, op):
    """Several 2048-point tiles and a ragged tail, heavy ties (few levels),
    many distinct values (odd and even rank bit counts: a one-level last
    pass), a lone datum; every result equals the oracle's."""
    rng = np.random.default_rng(900 + 10 * m + len(op) + len(dt))
    for nD, nQ, levels in ((5000, 4000, 30), (3001, 2999, 3000), (700, 9000, 6), (1, 5000, 3), (4100, 1, 50)):
        D, Q, w = workloads.random_small(rng, m, nD, nQ, levels, dt, wt)
        wv = None if op == "count" else w
        _check(D, Q, wv, op)


@pytest.mark.parametrize("m", [1, 2])
def test_wavelet_nonstrict_masks(m):
    rng = np.random.default_rng(950 + m)
    for mask in range(1 << m):
        for dt, wt, op in (("i32", "i64", "sum"), ("f32", "f32", "sum"), ("i32", "i32", "max")):
            D, Q, w = workloads.random_small(rng, m, 4500, 3500, 25, dt, wt)
            _check(D, Q, w, op, nonstrict=mask)


def test_wavelet_degenerate_cases():
    # all points equal: a single rank in every coordinate, every output e
    D = np.full((3000, 2), 7, np.int32)
    Q = np.full((2000, 2), 7, np.int32)
    w = np.arange(3000, dtype=np.int64)
    assert np.all(_fw(D, Q, w, "sum") == 0)
    assert np.all(_fw(D, Q, w, "sum", nonstrict=3) == w.sum())
    # no data: every output e
    Q = np.random.default_rng(3).integers(0, 100, size=(5000, 2)).astype(np.int32)
    got = _fw(np.zeros((0, 2), np.int32), Q, np.zeros(0, np.int32), "max")
    assert np.all(got == np.iinfo(np.int32).min)
    # one query above everything
    rng = np.random.default_rng(4)
    D = rng.integers(0, 1000, size=(6000, 2)).astype(np.int32)
    w = rng.integers(-1000, 1000, size=6000).astype(np.int64)
    assert _fw(D, np.array([[5000, 5000]], np.int32), w, "sum")[0] == w.sum()
    # the m = 1 case is a prefix scan along the coordinate
    x = rng.integers(0, 500, size=7000).astype(np.int32)
    q = rng.integers(0, 500, size=3000).astype(np.int32)
    wx = rng.integers(-1000, 1000, size=7000).astype(np.int64)
    order = np.argsort(x, kind="stable")
    cs = np.concatenate([[0], np.cumsum(wx[order])])
    want = cs[np.searchsorted(x[order], q, side="left")]
    assert np.array_equal(_fw(x[:, None], q[:, None], wx, "sum"), want)


def test_wavelet_equals_records_pipeline_at_scale():
    """|D| = |Q| = 2^20, the tied-float recipe: the level-wise passes give the
    int64 sums of the Sec. 5 pipeline bit for bit, float32 sums within the
    bound on sampled queries; the statistics report the passes."""
    p = workloads.tied_floats(n=1 << 20, weights="i32")
    w64 = p.w.astype(np.int64)
    a = _fw(p.D, p.Q, w64, "sum")
    st = domagg.stats()
    b = _fw(p.D, p.Q, w64, "sum", variant="improved")
    assert np.array_equal(a, b)
    assert st["n_records"] == 0 and st["record_passes"] == (st["rank_bits"][0] + 1) // 2
    assert np.array_equal(_fw(p.D, p.Q, p.w, "max"), _fw(p.D, p.Q, p.w, "max", variant="improved"))
    pf = workloads.tied_floats(n=1 << 20)
    got = _fw(pf.D, pf.Q, pf.w, "sum")
    qi = np.sort(np.random.default_rng(5).choice(1 << 20, 256, replace=False))
    assert_matches_oracle(got, pf.D, pf.Q, pf.w, "sum", qidx=qi)


def test_wavelet_rejects_m3():
    D = np.zeros((4, 3), np.int32)
    with pytest.raises(domagg.DomaggError) as e:
        _fw(D, D, np.ones(4, np.int64), "sum")
    assert e.value.status == 2


@pytest.mark.parametrize("m", [1, 2])
def test_wavelet_backward_and_autograd(m):
    """The adjoint by the level-wise formulation: grad_w[d] = sum of g[q] over
    q dominating d (every non-strict mask), against the oracle on the
    negated, role-swapped problem; the autograd function with variant
    "wavelet" gives the same gradient."""
    rng = np.random.default_rng(970 + m)
    for mask in range(1 << m):
        D, Q, _ = workloads.random_small(rng, m, 3500, 3000, 40, "f32", "f32")
        g = rng.standard_normal(3000).astype(np.float32)
        got = domagg.backward(to_dev(D), to_dev(Q), to_dev(g), nonstrict=mask, variant="wavelet").cpu().numpy()
        want, S = oracle.brute(-Q, -D, g, "sum", nonstrict=mask)
        assert_matches_oracle(got, -Q, -D, g, "sum", want=want, S=S)
    D, Q, w = workloads.random_small(rng, m, 2500, 2000, 300, "i32", "f32")
    c = rng.standard_normal(2000).astype(np.float32)
    wd = to_dev(w).requires_grad_(True)
    out = domagg.dominance_sum(to_dev(D), to_dev(Q), wd, 0, "wavelet")
    want_out, S_out = oracle.brute(D, Q, w, "sum")
    assert_matches_oracle(out.detach().cpu().numpy(), D, Q, w, "sum", want=want_out, S=S_out)
    (out * to_dev(c)).sum().backward()
    want, S = oracle.brute(-Q, -D, c, "sum")
    assert_matches_oracle(wd.grad.cpu().numpy(), -Q, -D, c, "sum", want=want, S=S)
    with pytest.raises(domagg.DomaggError) as e:
        domagg.backward(to_dev(D), to_dev(Q), to_dev(c), variant="basic")
    assert e.value.status == 2


def test_wavelet_full_size_integer_results_equal_records_pipeline():
    """At the full size (|D| = |Q| = 2^24, tied float coordinates) every one
    of the 2^24 integer results of the level-wise formulation equals the
    Sec. 5 record pipeline's: int64 sums, int32 max and the non-strict
    count (each path is checked against the oracle elsewhere)."""
    p = workloads.tied_floats(weights="i32")
    D, Q = to_dev(p.D), to_dev(p.Q)
    w64 = to_dev(p.w.astype(np.int64))
    w32 = to_dev(p.w)
    t = torch()
    for w, op, ns in ((w64, "sum", 0), (w32, "max", 0), (None, "count", 3)):
        a = domagg.forward(D, Q, w, op, nonstrict=ns, variant="wavelet")
        b = domagg.forward(D, Q, w, op, nonstrict=ns, variant="improved")
        t.cuda.synchronize()
        assert t.equal(a, b), op
