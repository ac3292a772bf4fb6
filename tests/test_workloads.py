"""The seeded input recipes (CPU): every workload has the shapes, ranges,
grids and tie structure its recipe states, and the same seed gives the same
arrays.  The recipes stand in for the data the paper never measures on."""
import numpy as np

from paper_2305_16751_gb300 import workloads


def test_small_int_recipe():
    p = workloads.small_int()
    assert p.D.shape == (4096, 2) and p.Q.shape == (4096, 2) and p.D.dtype == np.int32
    assert p.D.min() >= 0 and p.Q.max() < 2**20 and p.D.max() < 2**20
    assert p.w.dtype == np.int64 and p.w.min() >= -1000 and p.w.max() <= 1000
    q = workloads.small_int()
    assert np.array_equal(p.D, q.D) and np.array_equal(p.w, q.w)
    assert not np.array_equal(p.D, workloads.small_int(seed=1).D)


def test_tied_floats_recipe():
    n = 1 << 16
    p = workloads.tied_floats(n=n)
    for X in (p.D, p.Q):
        assert X.dtype == np.float32 and X.shape == (n, 2)
        assert X.min() >= 0.0 and X.max() < 1.0
        x64 = X.astype(np.float64)
        assert np.all(x64 * 2.0**24 == np.floor(x64 * 2.0**24))  # the 2^-24 grid
        on16 = np.all(x64 * 2.0**16 == np.floor(x64 * 2.0**16), axis=1)
        # the Bernoulli(0.25) quantised points, plus the few already on the coarse grid
        assert abs(on16.mean() - 0.25) < 0.01
    # ties inside and across D and Q
    assert len(np.unique(p.D[:, 0])) < n and len(np.intersect1d(p.D[:, 0], p.Q[:, 0])) > 0
    assert p.w.dtype == np.float32 and abs(p.w.mean()) < 0.02 and abs(p.w.std() - 1.0) < 0.02 and p.op == "sum"
    pm = workloads.tied_floats(n=n, weights="i32")
    assert pm.w.dtype == np.int32 and pm.op == "max"
    assert pm.w.min() >= -2**30 and pm.w.max() < 2**30


def test_gaussian_mixture_recipe():
    p = workloads.gaussian_mixture_i32(n=1 << 15)
    for X in (p.D, p.Q):
        assert X.dtype == np.int32 and X.shape == (1 << 15, 3)
        assert X.min() >= 0 and X.max() <= 2**24 - 1
    assert p.w.dtype == np.int64 and p.w.min() >= 0 and p.w.max() < 2**20
    # a mixture: the coordinates cluster (far fewer distinct 2^16-wide cells than uniform draws fill)
    cells = np.unique(p.D[:, 0] >> 16).size
    assert cells < 256


def test_autograd_and_ecdf_recipes():
    p = workloads.autograd_floats(n=4096)
    assert p.extra["c"].shape == (4096,) and p.w.dtype == np.float32
    x = p.D.astype(np.float64)
    assert np.all(x * 2.0**24 == np.floor(x * 2.0**24))
    e = workloads.ecdf_samples(n=4096, m=3, shift=0.5)
    y = e.D.astype(np.float64)
    assert np.all(y * 256.0 == np.round(y * 256.0))  # the 2^-8 grid
    assert e.Q.mean() > e.D.mean() + 0.3  # the shift of the second sample
    assert e.w is None and e.op == "count"


def test_batch_recipe():
    ms, sizes = workloads.batch_sizes()
    assert ms.shape == (4096,) and set(np.unique(ms)) == {2, 3} and abs((ms == 2).mean() - 0.5) < 0.03
    assert sizes.min() >= 256 and sizes.max() <= 2**18
    # log-uniform on [2^8, 2^18]: half the sizes below the geometric middle 2^13
    assert abs((sizes < 2**13).mean() - 0.5) < 0.03
    probs = workloads.batch_instances(k=6, lo=256, hi=1024)
    for p in probs:
        assert p.D.dtype == np.int32 and p.D.min() >= 0 and p.w.dtype == np.float32 and p.m in (2, 3)
        assert p.D.shape == p.Q.shape and p.D.shape[1] == p.m


def test_random_small_levels():
    rng = np.random.default_rng(0)
    D, Q, w = workloads.random_small(rng, 3, 500, 400, 7, "f32", "i64")
    vals = np.unique(np.concatenate([D, Q]))
    assert vals.size <= 8 and D.dtype == np.float32 and w.dtype == np.int64  # 2 * ceil(7 / 2) values
    assert np.all(vals * 2 == np.round(vals * 2))  # half-integers, negatives included
    assert vals.min() < 0
