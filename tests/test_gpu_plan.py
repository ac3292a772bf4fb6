"""Planned batches (domagg_batch_plan / domagg_plan_run): a run that neither
synchronises nor allocates, replayed from a CUDA graph with new buffer
contents, against the oracle and against the unplanned batch."""
import numpy as np
import pytest

from gpu_helpers import assert_matches_oracle, to_dev, torch
from paper_2305_16751_gb300 import domagg, workloads

pytestmark = pytest.mark.gpu


def _problems(rng, n, wt):
    """(D, Q, w) host arrays and the number of distinct coordinate values of
    each (mixed m, sizes and tie levels)."""
    probs, levels = [], []
    for i in range(n):
        m = 1 + i % 3
        nD, nQ = int(rng.integers(0, 2500)), int(rng.integers(1, 2500))
        lv = int(rng.integers(2, 400))
        probs.append(workloads.random_small(rng, m, nD, nQ, lv, "i32", wt))
        levels.append(lv)
    return probs, levels


def _refill(rng, dev_probs, host_probs, levels, wt):
    """New contents of the same shapes and tie levels (so of similar record
    counts), written in place."""
    new = []
    for (Dd, Qd, wd), (D, Q, w), lv in zip(dev_probs, host_probs, levels):
        D2, Q2, w2 = workloads.random_small(rng, D.shape[1], D.shape[0], Q.shape[0], lv, "i32", wt)
        Dd.copy_(to_dev(D2))
        Qd.copy_(to_dev(Q2))
        wd.copy_(to_dev(w2))
        new.append((D2, Q2, w2))
    return new


def test_plan_run_equals_unplanned_batch():
    rng = np.random.default_rng(901)
    probs, _ = _problems(rng, 30, "i64")
    dev = [(to_dev(D), to_dev(Q), to_dev(w)) for D, Q, w in probs]
    want = domagg.batch(dev, "sum")
    plan = domagg.BatchPlan(dev, "sum", headroom=0.5)
    try:
        for _ in range(2):
            plan.run()
            plan.status()
            for o, wv in zip(plan.outs, want):
                assert torch().equal(o, wv)
    finally:
        plan.close()


@pytest.mark.parametrize("op,wt", [("sum", "f32"), ("sum", "i64"), ("max", "i32"), ("count", "i64")])
def test_plan_graph_replay_with_new_data(op, wt):
    t = torch()
    rng = np.random.default_rng(902)
    host, levels = _problems(rng, 24, wt)
    dev = [(to_dev(D), to_dev(Q), to_dev(w)) for D, Q, w in host]
    plan = domagg.BatchPlan(dev, op, headroom=1.0)
    try:
        side = t.cuda.Stream()
        side.wait_stream(t.cuda.current_stream())
        g = t.cuda.CUDAGraph()
        with t.cuda.stream(side):
            with t.cuda.graph(g, stream=side):
                plan.run()
        t.cuda.synchronize()
        for _ in range(2):
            host = _refill(rng, dev, host, levels, wt)
            g.replay()
            plan.status()
            for (D, Q, w), o in zip(host, plan.outs):
                assert_matches_oracle(o.cpu().numpy(), D, Q, w if op != "count" else None, op)
    finally:
        plan.close()


def test_plan_capacity_exceeded_is_reported_and_recoverable():
    """Planned on data whose every first coordinate ties (no records for
    m >= 2), then run on spread-out data (50000 points: at m = 3 the three
    first-rank levels above the groups need records in HBM): the run reports
    DOMAGG_ERR_OOM and writes nothing out of bounds; back on tied data it is
    correct again."""
    t = torch()
    rng = np.random.default_rng(903)
    host = []
    for m in (2, 3):
        D = np.full((30000, m), 7, dtype=np.int32)
        Q = np.full((20000, m), 9, dtype=np.int32)
        w = rng.integers(-50, 50, size=30000).astype(np.int64)
        host.append((D, Q, w))
    dev = [(to_dev(D), to_dev(Q), to_dev(w)) for D, Q, w in host]
    plan = domagg.BatchPlan(dev, "sum", headroom=0.0)
    try:
        for (D, Q, w), o in zip(host, plan.outs):
            assert_matches_oracle(o.cpu().numpy(), D, Q, w, "sum")
        for Dd, Qd, _ in dev:
            Dd.copy_(t.randint(0, 1 << 20, Dd.shape, dtype=t.int32, device="cuda"))
            Qd.copy_(t.randint(0, 1 << 20, Qd.shape, dtype=t.int32, device="cuda"))
        plan.run()
        with pytest.raises(domagg.DomaggError) as ei:
            plan.status()
        assert ei.value.status == 3  # DOMAGG_ERR_OOM
        for (D, Q, _), (Dd, Qd, _) in zip(host, dev):
            Dd.copy_(to_dev(D))
            Qd.copy_(to_dev(Q))
        plan.run()
        plan.status()
        for (D, Q, w), o in zip(host, plan.outs):
            assert_matches_oracle(o.cpu().numpy(), D, Q, w, "sum")
    finally:
        plan.close()


def test_plan_batch_workload_shape():
    """The batch workload (uniform int32 coordinates, float32 weights) at
    reduced instance count and sizes, replayed from a graph."""
    t = torch()
    probs = workloads.batch_instances(k=48, lo=64, hi=4096)
    dev = [(to_dev(p.D), to_dev(p.Q), to_dev(p.w)) for p in probs]
    plan = domagg.BatchPlan(dev, "sum", headroom=0.1)
    try:
        side = t.cuda.Stream()
        side.wait_stream(t.cuda.current_stream())
        g = t.cuda.CUDAGraph()
        with t.cuda.stream(side):
            with t.cuda.graph(g, stream=side):
                plan.run()
        for o in plan.outs:
            o.fill_(float("nan"))
        g.replay()
        plan.status()
        for p, o in zip(probs, plan.outs):
            assert_matches_oracle(o.cpu().numpy(), p.D, p.Q, p.w, "sum")
    finally:
        plan.close()


def test_plan_autotune_keeps_results():
    """The autotuner times nine launch shapes and keeps the fastest; runs
    after it give the same (integer) results as the unplanned batch."""
    rng = np.random.default_rng(904)
    probs, _ = _problems(rng, 20, "i64")
    dev = [(to_dev(D), to_dev(Q), to_dev(w)) for D, Q, w in probs]
    want = domagg.batch(dev, "sum")
    plan = domagg.BatchPlan(dev, "sum", headroom=0.2)
    try:
        ms = plan.autotune()
        assert ms > 0
        plan.run()
        plan.status()
        for o, wv in zip(plan.outs, want):
            assert torch().equal(o, wv)
    finally:
        plan.close()


def test_plan_autotune_with_ranges_of_top_levels():
    """m = 2 instances large enough that the top levels run in hundreds of
    ranges of tiles (8.5e6 points in 690 tiles): the range table, uploaded
    by the plan's measuring run, does not depend on the launch shapes the
    autotuner tries, and runs after it give the unplanned batch's integer
    sums."""
    rng = np.random.default_rng(905)
    probs = [workloads.random_small(rng, 2, n, n, 1 << 22, "i32", "i64") for n in (2_500_000, 1_700_000, 40_000)]
    dev = [(to_dev(D), to_dev(Q), to_dev(w)) for D, Q, w in probs]
    want = domagg.batch(dev, "sum")
    plan = domagg.BatchPlan(dev, "sum", headroom=0.2)
    try:
        plan.autotune()
        for _ in range(2):
            plan.run()
            plan.status()
            for o, wv in zip(plan.outs, want):
                assert torch().equal(o, wv)
    finally:
        plan.close()


def test_plan_with_both_key_classes_and_m4():
    """Planned runs with m = 3 instances large enough that some levels need
    64-bit node keys (the rest 32-bit), and m = 4 instances, replayed from a
    graph with new contents."""
    t = torch()
    rng = np.random.default_rng(905)
    host, levels = [], []
    for m, nD, nQ, lv in ((3, 40000, 40000, 60000), (4, 3000, 2500, 50), (3, 500, 700, 20), (2, 30000, 30000, 9000)):
        host.append(workloads.random_small(rng, m, nD, nQ, lv, "i32", "i64"))
        levels.append(lv)
    dev = [(to_dev(D), to_dev(Q), to_dev(w)) for D, Q, w in host]
    plan = domagg.BatchPlan(dev, "sum", headroom=0.5)
    try:
        for (D, Q, w), o in zip(host, plan.outs):
            qi = np.sort(rng.choice(Q.shape[0], min(Q.shape[0], 300), replace=False))
            assert_matches_oracle(o.cpu().numpy(), D, Q, w, "sum", qidx=qi)
        side = t.cuda.Stream()
        side.wait_stream(t.cuda.current_stream())
        g = t.cuda.CUDAGraph()
        with t.cuda.stream(side):
            with t.cuda.graph(g, stream=side):
                plan.run()
        host = _refill(rng, dev, host, levels, "i64")
        g.replay()
        plan.status()
        for (D, Q, w), o in zip(host, plan.outs):
            qi = np.sort(rng.choice(Q.shape[0], min(Q.shape[0], 300), replace=False))
            assert_matches_oracle(o.cpu().numpy(), D, Q, w, "sum", qidx=qi)
    finally:
        plan.close()


def test_plan_with_overflowing_groups():
    """Instances whose first coordinate piles 11000 points on one value: the
    group holding them overflows shared memory, so only those points' deep
    levels go through the planned record workspace (m = 2 and m = 3, beside
    instances without such a tie); the planned run equals the oracle."""
    rng = np.random.default_rng(904)
    host = []
    for m in (2, 3, 2, 3):
        D, Q, w = workloads.random_small(rng, m, 40000, 31000, 1 << 20, "i32", "i64")
        if len(host) < 2:
            D[:6000, 0] = 0
            Q[:5000, 0] = 0
        host.append((D, Q, w))
    dev = [(to_dev(D), to_dev(Q), to_dev(w)) for D, Q, w in host]
    plan = domagg.BatchPlan(dev, "sum", headroom=0.1)
    try:
        for _ in range(2):
            plan.run()
            plan.status()
            for (D, Q, w), o in zip(host, plan.outs):
                assert_matches_oracle(o.cpu().numpy(), D, Q, w, "sum")
    finally:
        plan.close()
