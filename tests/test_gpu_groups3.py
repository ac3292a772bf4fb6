"""The m = 3 deep first-rank levels taken per group of ranks in shared
memory (k_group3) against the same pipeline with every level's records in
HBM (tuning knob group_bits = 0), and both against the oracle: every op,
ties, every group width, groups too large for shared memory, non-strict
coordinates, the backward pass, batches and shards."""
import contextlib

import numpy as np
import pytest

import oracle
from gpu_helpers import assert_matches_oracle, gpu_forward, to_dev, torch
from paper_2305_16751_gb300 import domagg, workloads

pytestmark = pytest.mark.gpu


@contextlib.contextmanager
def group_bits(v):
    h = domagg.handle(0)
    domagg.domagg_set_tuning(h, "group_bits", v)
    try:
        yield
    finally:
        domagg.domagg_set_tuning(h, "group_bits", 13)


CASES = [("i32", "i64", "sum"), ("f32", "i32", "max"), ("f32", "i64", "count"), ("i32", "i32", "min"),
         ("f32", "f32", "sum"), ("i32", "f32", "max"), ("f32", "f32", "min")]
SIZES = ((12000, 9000, 1 << 20), (9001, 7003, 5000), (15000, 14000, 300), (1, 5000, 50), (5000, 1, 7),
         (3000, 3000, 2), (20000, 3000, 1 << 12))


@pytest.mark.parametrize("dt,wt,op", CASES)
def test_groups3_equal_records_in_hbm(dt, wt, op):
    rng = np.random.default_rng(6100 + len(op) + len(wt) + len(dt))
    for nD, nQ, levels in SIZES:
        D, Q, w = workloads.random_small(rng, 3, nD, nQ, levels, dt, wt)
        wv = None if op == "count" else w
        got = gpu_forward(D, Q, wv, op)
        st = domagg.stats()
        assert st["n_records"] == oracle.record_count(D, Q)
        if levels >= 300:
            assert st["n_records_shared"] > 0, (nD, nQ, levels)
        with group_bits(0):
            ref = gpu_forward(D, Q, wv, op)
            assert domagg.stats()["n_records_shared"] == 0
        assert_matches_oracle(got, D, Q, wv, op)
        if not (op == "sum" and wt == "f32"):
            assert np.array_equal(got, ref), (nD, nQ, levels)


def test_every_group3_width_gives_the_same_sums():
    rng = np.random.default_rng(6200)
    D, Q, w = workloads.random_small(rng, 3, 12000, 10000, 1 << 16, "i32", "i64")
    want, _ = oracle.brute(D, Q, w, "sum")
    shared = []
    for g in range(0, 14):
        with group_bits(g):
            got = gpu_forward(D, Q, w, "sum")
            shared.append(domagg.stats()["n_records_shared"])
        assert np.array_equal(got, want), g
    assert shared[0] == 0 and all(b >= a for a, b in zip(shared, shared[1:])) and shared[13] > 0


def test_groups3_heavy_ties():
    """Few distinct first coordinates: groups too large for shared memory
    (every level through HBM); few distinct second coordinates (a handful
    of local second-rank levels); a single second coordinate (no records)."""
    rng = np.random.default_rng(6300)
    D, Q, w = workloads.random_small(rng, 3, 15000, 15000, 3, "i32", "i64")
    got = gpu_forward(D, Q, w, "sum")
    assert domagg.stats()["n_records_shared"] == 0
    assert_matches_oracle(got, D, Q, w, "sum")
    D[:, 0] = rng.integers(0, 1 << 20, size=15000)
    Q[:, 0] = rng.integers(0, 1 << 20, size=15000)
    got = gpu_forward(D, Q, w, "sum")
    assert domagg.stats()["n_records_shared"] > 0
    assert_matches_oracle(got, D, Q, w, "sum")
    D[:, 1] = 7
    Q[:, 1] = 7
    got = gpu_forward(D, Q, w, "sum")
    assert np.array_equal(got, np.zeros_like(got))
    D[:, 1] = rng.integers(0, 600, size=15000)
    Q[:, 1] = rng.integers(0, 600, size=15000)
    D[:, 0] = rng.integers(0, 600, size=15000)
    Q[:, 0] = rng.integers(0, 600, size=15000)
    got = gpu_forward(D, Q, w, "sum")
    st = domagg.stats()
    assert 0 < st["n_records_shared"] < st["n_records"]
    assert_matches_oracle(got, D, Q, w, "sum")


@pytest.mark.parametrize("mask", [1, 2, 3, 4, 5, 6, 7])
def test_groups3_nonstrict(mask):
    rng = np.random.default_rng(6400 + mask)
    D, Q, w = workloads.random_small(rng, 3, 9000, 8000, 2000, "f32", "i64")
    got = domagg.forward(to_dev(D), to_dev(Q), to_dev(w), "sum", nonstrict=mask).cpu().numpy()
    torch().cuda.synchronize()
    assert domagg.stats()["n_records_shared"] > 0
    want, _ = oracle.brute(D, Q, w, "sum", nonstrict=mask)
    assert np.array_equal(got, want)


def test_groups3_backward():
    rng = np.random.default_rng(6500)
    D, Q, _ = workloads.random_small(rng, 3, 7000, 6000, 4000, "i32", "i64")
    # integer gradients below 2^24 in every sum: float32 results are exact
    g = rng.integers(-1000, 1001, size=6000).astype(np.float32)
    got = domagg.backward(to_dev(D), to_dev(Q), to_dev(g)).cpu().numpy()
    torch().cuda.synchronize()
    want, _ = oracle.brute_transpose(D, Q, g)
    assert np.array_equal(got.astype(np.float64), want)


def test_groups3_in_a_batch():
    """m = 3 instances of very different sizes in one batch: some with
    groups, some too small or too tied for them, some empty."""
    rng = np.random.default_rng(6600)
    probs = []
    for nD, nQ, levels in ((9000, 7000, 1 << 16), (1, 1, 2), (0, 300, 10), (3000, 0, 10), (777, 555, 3),
                           (15000, 14000, 1 << 20), (6000, 5000, 5)):
        D, Q, w = workloads.random_small(rng, 3, max(nD, 1), max(nQ, 1), levels, "i32", "i64")
        probs.append((D[:nD], Q[:nQ], w[:nD]))
    for gb in (13, 0):
        with group_bits(gb):
            outs = domagg.batch([(to_dev(D), to_dev(Q), to_dev(w)) for D, Q, w in probs], "sum")
            torch().cuda.synchronize()
        for (D, Q, w), o in zip(probs, outs):
            if Q.shape[0] == 0:
                continue
            want, _ = oracle.brute(D, Q, w, "sum")
            assert np.array_equal(o.cpu().numpy(), want), (gb, D.shape, Q.shape)


@pytest.mark.parametrize("nshards", [2, 3])
def test_groups3_shards(nshards):
    """Shards split the groups and the levels above them; F over the shards'
    outputs is the whole result."""
    rng = np.random.default_rng(6700 + nshards)
    D, Q, w = workloads.random_small(rng, 3, 9000, 8000, 1 << 14, "i32", "i64")
    want, _ = oracle.brute(D, Q, w, "sum")
    total = np.zeros(Q.shape[0], dtype=np.int64)
    for sh in range(nshards):
        part, _ = domagg.forward_shard(to_dev(D), to_dev(Q), to_dev(w), "sum", sh, nshards)
        torch().cuda.synchronize()
        total += part.cpu().numpy().astype(np.int64)
    assert np.array_equal(total, want)


@pytest.mark.parametrize("m,top", [(2, 0), (2, 12), (3, 12)])
def test_overflowing_groups_go_through_hbm(m, top):
    """A first coordinate with 11000 points on one value (as where a
    distribution is clipped): the group holding it is too large for shared
    memory, so its points' levels below gS go through the records in HBM
    while every other group stays in shared memory (m = 2 with and without
    the top-level tiles, m = 3)."""
    rng = np.random.default_rng(6800 + m + top)
    D, Q, w = workloads.random_small(rng, m, 40000, 31000, 1 << 20, "i32", "i64")
    D[:6000, 0] = 0
    Q[:5000, 0] = 0
    h = domagg.handle(0)
    domagg.domagg_set_tuning(h, "top_bits", top)
    try:
        got = gpu_forward(D, Q, w, "sum")
        st = domagg.stats()
    finally:
        domagg.domagg_set_tuning(h, "top_bits", 12)
    want, _ = oracle.brute(D, Q, w, "sum")
    assert np.array_equal(got, want)
    assert st["n_records"] == oracle.record_count(D, Q)
    assert 0 < st["n_records_shared"] < st["n_records"]
