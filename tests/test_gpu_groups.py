"""The m = 2 deep rank levels taken per group of ranks in shared memory
(k_group) against the same pipeline with every level's records in HBM
(tuning knob group_bits = 0; the top levels' tiles are off here), and both
against the oracle."""
import contextlib

import numpy as np
import pytest

import oracle
from gpu_helpers import assert_matches_oracle, gpu_forward, to_dev, torch
from paper_2305_16751_gb300 import domagg, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def records_above_the_groups():
    """These tests compare the groups with the records in HBM: the levels
    above the groups go through the records too (top_bits = 0)."""
    h = domagg.handle(0)
    domagg.domagg_set_tuning(h, "top_bits", 0)
    yield
    domagg.domagg_set_tuning(h, "top_bits", 12)


@contextlib.contextmanager
def group_bits(v):
    h = domagg.handle(0)
    domagg.domagg_set_tuning(h, "group_bits", v)
    try:
        yield
    finally:
        domagg.domagg_set_tuning(h, "group_bits", 13)


CASES = [("i32", "i64", "sum"), ("f32", "i32", "max"), ("f32", "i64", "count"), ("i32", "i32", "min"),
         ("f32", "f32", "sum")]


@pytest.mark.parametrize("dt,wt,op", CASES)
def test_groups_equal_records_in_hbm(dt, wt, op):
    rng = np.random.default_rng(4100 + len(op) + len(wt))
    for nD, nQ, levels in ((30000, 20000, 1 << 20), (9001, 7003, 5000), (40000, 35000, 300), (1, 5000, 50)):
        D, Q, w = workloads.random_small(rng, 2, nD, nQ, levels, dt, wt)
        wv = None if op == "count" else w
        got = gpu_forward(D, Q, wv, op)
        st = domagg.stats()
        assert st["n_records"] == oracle.record_count(D, Q)
        with group_bits(0):
            ref = gpu_forward(D, Q, wv, op)
            assert domagg.stats()["n_records_shared"] == 0
        assert_matches_oracle(got, D, Q, wv, op)
        if not (op == "sum" and wt == "f32"):
            assert np.array_equal(got, ref)


def test_every_group_width_gives_the_same_sums():
    rng = np.random.default_rng(4200)
    D, Q, w = workloads.random_small(rng, 2, 20000, 18000, 1 << 16, "i32", "i64")
    want, _ = oracle.brute(D, Q, w, "sum")
    shared = []
    for g in range(0, 14):
        with group_bits(g):
            got = gpu_forward(D, Q, w, "sum")
            shared.append(domagg.stats()["n_records_shared"])
        assert np.array_equal(got, want), g
    assert shared[0] == 0 and all(b >= a for a, b in zip(shared, shared[1:])) and shared[13] > 0


def test_heavy_ties_fall_back_to_records_in_hbm():
    """Groups that would exceed the shared-memory capacity: with 3 distinct
    first coordinates over 60000 points even 2-rank groups are too large, so
    every level goes through HBM; with 600 distinct values a narrower group
    width is chosen."""
    rng = np.random.default_rng(4300)
    D, Q, w = workloads.random_small(rng, 2, 30000, 30000, 3, "i32", "i64")
    got = gpu_forward(D, Q, w, "sum")
    assert domagg.stats()["n_records_shared"] == 0
    assert_matches_oracle(got, D, Q, w, "sum")
    D[:, 1] = rng.integers(0, 1 << 20, size=30000)
    Q[:, 1] = rng.integers(0, 1 << 20, size=30000)
    D[:, 0] = rng.integers(0, 600, size=30000)
    Q[:, 0] = rng.integers(0, 600, size=30000)
    got = gpu_forward(D, Q, w, "sum")
    st = domagg.stats()
    assert 0 < st["n_records_shared"] < st["n_records"]
    assert_matches_oracle(got, D, Q, w, "sum")


@pytest.mark.parametrize("mask", [1, 2, 3])
def test_groups_with_nonstrict_coordinates(mask):
    rng = np.random.default_rng(4400 + mask)
    D, Q, w = workloads.random_small(rng, 2, 25000, 22000, 2000, "f32", "i64")
    got = domagg.forward(to_dev(D), to_dev(Q), to_dev(w), "sum", nonstrict=mask).cpu().numpy()
    torch().cuda.synchronize()
    assert domagg.stats()["n_records_shared"] > 0
    want, _ = oracle.brute(D, Q, w, "sum", nonstrict=mask)
    assert np.array_equal(got, want)


def test_integer_results_repeat_exactly():
    """Five forward calls on the same 2^20-per-side tied input give the same
    integer results as the oracle every time (a race between tiles or groups
    would show as a run-to-run difference)."""
    p = workloads.tied_floats(n=1 << 20, weights="i32")
    w64 = p.w.astype(np.int64)
    want_c, _ = oracle.sweep2(p.D, p.Q, None, "count", nonstrict=3)
    want_s, _ = oracle.sweep2(p.D, p.Q, w64, "sum")
    D, Q, w = to_dev(p.D), to_dev(p.Q), to_dev(w64)
    for _ in range(5):
        c = domagg.forward(D, Q, None, "count", nonstrict=3).cpu().numpy()
        s = domagg.forward(D, Q, w, "sum").cpu().numpy()
        assert np.array_equal(c, want_c) and np.array_equal(s, want_s)
