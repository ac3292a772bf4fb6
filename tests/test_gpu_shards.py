"""The forward split into shards (domagg_forward_shard) and joined by F
(domagg_combine): the flat map's records partitioned by node (rank levels of
the first coordinate, and groups of ranks for the levels taken in shared
memory), every shard after the same point phase.  The shards of one
problem, run one after the other on one GPU and joined, equal the whole
forward and the oracle, for 1 to 4 shards, m = 1, 2, 3 and every op.  For
m = 1 the flat map has one level and one node, so shard 0 takes all of it
and the other shards return the unit."""
import numpy as np
import pytest

import oracle
from gpu_helpers import assert_matches_oracle, gpu_forward, to_dev, torch
from paper_2305_16751_gb300 import domagg, workloads

pytestmark = pytest.mark.gpu


def _sharded(D, Q, w, op, nshards):
    t = torch()
    Dd, Qd, wd = to_dev(D), to_dev(Q), to_dev(w)
    parts, los = [], []
    for s in range(nshards):
        o, lo = domagg.forward_shard(Dd, Qd, wd, op, s, nshards)
        parts.append(o)
        los.append(lo)
    out = domagg.combine(parts, los if los[0] is not None else None, op, None if wd is None else wd.dtype)
    t.cuda.synchronize()
    return out.cpu().numpy(), [p.cpu().numpy() for p in parts]


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("op,wt", [("sum", "i64"), ("max", "i32"), ("count", "i64"), ("min", "f32")])
def test_shards_join_to_the_forward(m, op, wt):
    rng = np.random.default_rng(600 + m + len(op))
    D, Q, w = workloads.random_small(rng, m, 20000, 15000, 5000, "f32", wt)
    wv = None if op == "count" else w
    whole = gpu_forward(D, Q, wv, op)
    for ns in (1, 2, 3, 4):
        got, parts = _sharded(D, Q, wv, op, ns)
        assert np.array_equal(got, whole), (m, op, ns)
        if ns > 1 and op in ("sum", "count"):
            busy = sum(int(np.abs(p).sum() > 0) for p in parts)
            assert busy >= 2 if m >= 2 else busy == 1  # the work is split (m = 1: one level)
    assert_matches_oracle(got, D, Q, wv, op)


def test_shards_of_a_float32_sum_keep_float_float_pairs():
    """float32 sums: each shard returns its partials as float-float pairs, so
    joining 1..4 shards stays within the forward's tolerance of the exact sum
    (the groups of ranks in shared memory and the top levels are split
    between the shards)."""
    p = workloads.tied_floats(n=1 << 19)
    want, S = oracle.sweep2(p.D, p.Q, p.w, "sum")
    for ns in (1, 2, 4):
        got, _ = _sharded(p.D, p.Q, p.w, "sum", ns)
        assert_matches_oracle(got, p.D, p.Q, p.w, "sum", want=want, S=S)


def test_shard_arguments_are_checked():
    D = to_dev(np.zeros((4, 2), np.float32))
    w = to_dev(np.ones(4, np.float32))
    for shard, ns in ((2, 2), (-1, 2), (0, 0), (0, 65)):
        with pytest.raises(domagg.DomaggError) as e:
            domagg.forward_shard(D, D, w, "sum", shard, ns)
        assert e.value.status == 1
