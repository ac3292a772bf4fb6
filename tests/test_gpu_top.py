"""The m = 2 top rank levels per range of tiles in the order of the last
coordinate (k_top, k_top_carry, k_reduce_top) against the same pipeline with
those levels' records in HBM (tuning knob top_bits = 0), and both against the
oracle: every op, top widths 1 .. 12, with and without the groups below,
ranges of one and of many tiles (the carries across ranges), heavy ties (few
levels, a single node), non-strict coordinates and batches."""
import contextlib

import numpy as np
import pytest

import oracle
from gpu_helpers import assert_matches_oracle, gpu_forward, to_dev, torch
from paper_2305_16751_gb300 import domagg, workloads

pytestmark = pytest.mark.gpu


@contextlib.contextmanager
def knobs(**kv):
    h = domagg.handle(0)
    for k, v in kv.items():
        domagg.domagg_set_tuning(h, k, v)
    try:
        yield
    finally:
        domagg.domagg_set_tuning(h, "top_bits", 12)
        domagg.domagg_set_tuning(h, "group_bits", 13)
        domagg.domagg_set_tuning(h, "ranges_per_cta", 4)


CASES = [("i32", "i64", "sum"), ("f32", "i32", "max"), ("f32", "i64", "count"), ("i32", "i32", "min"),
         ("f32", "f32", "sum"), ("i32", "f32", "min"), ("f32", "f32", "max")]
SIZES = ((30000, 20000, 1 << 20), (9001, 7003, 5000), (40000, 35000, 300), (1, 5000, 50), (5000, 1, 7),
         (70000, 65000, 1 << 24), (3000, 3000, 2))


@pytest.mark.parametrize("gbits", [13, 0])
@pytest.mark.parametrize("dt,wt,op", CASES)
def test_top_levels_equal_records_in_hbm(dt, wt, op, gbits):
    rng = np.random.default_rng(5100 + len(op) + len(wt) + gbits)
    for nD, nQ, levels in SIZES:
        D, Q, w = workloads.random_small(rng, 2, nD, nQ, levels, dt, wt)
        wv = None if op == "count" else w
        with knobs(group_bits=gbits):
            got = gpu_forward(D, Q, wv, op)
            st = domagg.stats()
            with knobs(top_bits=0, group_bits=gbits):
                ref = gpu_forward(D, Q, wv, op)
                st0 = domagg.stats()
        assert st["n_records"] == st0["n_records"] == oracle.record_count(D, Q)
        assert st["n_records_shared"] >= st0["n_records_shared"]
        want, S = oracle.sweep2(D, Q, wv, op)
        assert_matches_oracle(got, D, Q, wv, op, want=want, S=S)
        if not (op == "sum" and wt == "f32"):
            assert np.array_equal(got, ref)


def test_every_top_width_and_many_ranges():
    """Top widths 1 .. 12 over 130000 points in ranges of one tile (the
    nodes' carries cross ten range boundaries) give the oracle's integer
    sums, without groups and with them, for two range targets."""
    rng = np.random.default_rng(5200)
    D, Q, w = workloads.random_small(rng, 2, 70000, 60000, 1 << 18, "i32", "i64")
    want, _ = oracle.sweep2(D, Q, w, "sum")
    for gbits in (0, 13):
        for rpc in (1, 64):
            shared = []
            for tb in range(0, 13):
                with knobs(top_bits=tb, group_bits=gbits, ranges_per_cta=rpc):
                    got = gpu_forward(D, Q, w, "sum")
                    shared.append(domagg.stats()["n_records_shared"])
                assert np.array_equal(got, want), (gbits, rpc, tb)
            assert all(b >= a for a, b in zip(shared, shared[1:])) and shared[12] > shared[0]


@pytest.mark.parametrize("mask", [1, 2, 3])
def test_top_levels_nonstrict(mask):
    rng = np.random.default_rng(5300 + mask)
    D, Q, w = workloads.random_small(rng, 2, 25000, 22000, 2000, "f32", "i64")
    want, _ = oracle.sweep2(D, Q, w, "sum", nonstrict=mask)
    for gbits in (13, 0):
        with knobs(group_bits=gbits, ranges_per_cta=64):
            got = domagg.forward(to_dev(D), to_dev(Q), to_dev(w), "sum", nonstrict=mask).cpu().numpy()
            torch().cuda.synchronize()
        assert np.array_equal(got, want), gbits


def test_top_levels_in_a_batch():
    """Instances of very different sizes share the range table; some take
    several ranges (carries), some one, some have no top level at all."""
    rng = np.random.default_rng(5400)
    probs = []
    for nD, nQ, levels in ((20000, 15000, 1 << 16), (1, 1, 2), (0, 300, 10), (3000, 0, 10), (777, 555, 3),
                           (150000, 140000, 1 << 20), (60000, 50000, 5)):
        D, Q, w = workloads.random_small(rng, 2, max(nD, 1), max(nQ, 1), levels, "i32", "i64")
        probs.append((D[:nD], Q[:nQ], w[:nD]))
    for gbits in (13, 0):
        with knobs(group_bits=gbits, ranges_per_cta=64):
            outs = domagg.batch([(to_dev(D), to_dev(Q), to_dev(w)) for D, Q, w in probs], "sum")
            torch().cuda.synchronize()
        for (D, Q, w), o in zip(probs, outs):
            if Q.shape[0] == 0:
                continue
            want, _ = oracle.sweep2(D, Q, w, "sum")
            assert np.array_equal(o.cpu().numpy(), want), (gbits, D.shape, Q.shape)


def test_top_levels_at_2_20_repeat_exactly():
    """2^20 points per side with ties: integer sums equal the oracle's sweep
    and float32 sums are bit-identical on three consecutive calls (the
    carries are combined in a fixed order)."""
    p = workloads.tied_floats(n=1 << 20, weights="i32")
    w64 = p.w.astype(np.int64)
    want, _ = oracle.sweep2(p.D, p.Q, w64, "sum")
    D, Q, w, wf = to_dev(p.D), to_dev(p.Q), to_dev(w64), to_dev(p.w.astype(np.float32))
    for rpc in (4, 64):
        with knobs(ranges_per_cta=rpc):
            first = None
            for _ in range(3):
                got = domagg.forward(D, Q, w, "sum").cpu().numpy()
                assert np.array_equal(got, want), rpc
                f = domagg.forward(D, Q, wf, "sum").cpu().numpy()
                if first is None:
                    first = f
                assert np.array_equal(f.view(np.uint32), first.view(np.uint32)), rpc
