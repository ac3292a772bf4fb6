"""Forward parity of the CUDA path (through the C ABI) against the CPU oracle."""
import numpy as np
import pytest

import oracle
from gpu_helpers import assert_matches_oracle, gpu_forward, to_dev, torch
from paper_2305_16751_gb300 import domagg, workloads

pytestmark = pytest.mark.gpu


def test_small_int_workload_sum_and_count():
    """m=2, |D|=|Q|=4096, int32 coordinates in [0, 2^20), int64 weights."""
    p = workloads.small_int()
    for op in ("sum", "count"):
        got = gpu_forward(p.D, p.Q, p.w, op)
        assert_matches_oracle(got, p.D, p.Q, p.w if op == "sum" else None, op)


def test_record_count_equals_oracle_flat_map():
    p = workloads.small_int()
    gpu_forward(p.D, p.Q, p.w, "sum")
    st = domagg.stats()
    assert st["n_records"] == oracle.record_count(p.D, p.Q)
    assert st["n_points"] == 8192


CASES = [(m, dt, wt, op) for m in (1, 2, 3) for dt in ("i32", "f32")
         for wt, op in (("i64", "sum"), ("f32", "sum"), ("i32", "max"), ("f32", "max"), ("i64", "count"),
                        ("i32", "min"), ("f32", "min"))]


@pytest.mark.parametrize("m,dt,wt,op", CASES)
def test_random_tied_several_tiles(m, dt, wt, op):
    """Heavy ties (few distinct levels), several tiles and a ragged tail."""
    rng = np.random.default_rng(100 * m + len(dt) + len(op))
    for nD, nQ, levels in ((9001, 7003, 40), (5000, 6000, 3000), (3, 20000, 7)):
        D, Q, w = workloads.random_small(rng, m, nD, nQ, levels, dt, wt)
        got = gpu_forward(D, Q, w if op != "count" else None, op)
        assert_matches_oracle(got, D, Q, w if op != "count" else None, op)
        if op == "sum" and m >= 2:
            assert domagg.stats()["n_records"] == oracle.record_count(D, Q)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_sortscan_oracle_agrees(m):
    rng = np.random.default_rng(9 + m)
    D, Q, w = workloads.random_small(rng, m, 3000, 2500, 200, "i32", "i64")
    got = gpu_forward(D, Q, w, "sum")
    want, _ = oracle.sortscan(D, Q, w, "sum")
    assert np.array_equal(got, want)


def test_empty_data_gives_unit():
    Q = np.arange(20, dtype=np.int32).reshape(10, 2)
    D = np.zeros((0, 2), np.int32)
    assert gpu_forward(D, Q, np.zeros(0, np.int64), "sum").tolist() == [0] * 10
    assert gpu_forward(D, Q, np.zeros(0, np.int32), "max").tolist() == [np.iinfo(np.int32).min] * 10
    out = gpu_forward(D.astype(np.float32), Q.astype(np.float32), np.zeros(0, np.float32), "max")
    assert np.all(np.isneginf(out))


def test_empty_queries():
    D = np.arange(20, dtype=np.int32).reshape(10, 2)
    Q = np.zeros((0, 2), np.int32)
    assert gpu_forward(D, Q, np.ones(10, np.int64), "sum").shape == (0,)


def test_single_points_and_strictness():
    D = np.array([[1, 1], [1, 0], [0, 1], [0, 0]], np.int32)
    Q = np.array([[1, 1], [2, 2], [0, 0]], np.int32)
    w = np.array([1, 10, 100, 1000], np.int64)
    assert gpu_forward(D, Q, w, "sum").tolist() == [1000, 1111, 0]
    assert gpu_forward(D[:1], Q[1:2], w[:1], "sum").tolist() == [1]


def test_all_points_equal():
    D = np.full((5000, 3), 7, np.int32)
    Q = np.full((4000, 3), 7, np.int32)
    assert gpu_forward(D, Q, np.ones(5000, np.int64), "sum").tolist() == [0] * 4000
    assert domagg.stats()["n_records"] == 0


def test_signed_zero_and_infinities():
    D = np.array([[-0.0, 1.0], [-np.inf, -np.inf], [1.0, np.inf]], np.float32)
    Q = np.array([[0.0, 2.0], [0.5, 2.0], [np.inf, np.inf], [0.0, 0.0]], np.float32)
    w = np.array([3, 1, 10], np.int64)
    want, _ = oracle.brute(D, Q, w, "sum")
    assert gpu_forward(D, Q, w, "sum").tolist() == want.tolist() == [1, 4, 4, 1]


def test_nan_coordinate_is_reported():
    D = np.array([[np.nan, 1.0]], np.float32)
    Q = np.array([[1.0, 1.0]], np.float32)
    with pytest.raises(domagg.DomaggError) as e:
        gpu_forward(D, Q, np.ones(1, np.float32), "sum")
    assert e.value.name == "NAN"
    # the handle stays usable
    assert gpu_forward(np.zeros((1, 2), np.float32), np.ones((1, 2), np.float32), np.ones(1, np.float32),
                       "sum").tolist() == [1.0]


def test_int64_sum_wraps_and_int32_min():
    D = np.array([[0, 0], [1, 1]], np.int32)
    Q = np.array([[5, 5]], np.int32)
    assert gpu_forward(D, Q, np.array([2**62, 2**62], np.int64) * 2, "sum").tolist() == [0]
    assert gpu_forward(D, Q, np.array([-2**31, -2**31], np.int32), "max").tolist() == [-2**31]


def test_negative_and_extreme_int_coordinates():
    rng = np.random.default_rng(4)
    for m in (2, 3):
        D = rng.integers(-2**31, 2**31, size=(3000, m), dtype=np.int64).astype(np.int32)
        Q = rng.integers(-2**31, 2**31, size=(3000, m), dtype=np.int64).astype(np.int32)
        D[:10] = -2**31
        Q[:10] = 2**31 - 1
        w = rng.integers(-1000, 1000, size=3000, dtype=np.int64)
        assert_matches_oracle(gpu_forward(D, Q, w, "sum"), D, Q, w, "sum")


def test_deterministic_float_sum():
    p = workloads.tied_floats(n=50000)
    a = gpu_forward(p.D, p.Q, p.w, "sum")
    b = gpu_forward(p.D, p.Q, p.w, "sum")
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert_matches_oracle(a, p.D, p.Q, p.w, "sum")


def test_forward_host_matches_device():
    t = torch()
    p = workloads.tied_floats(n=30000)
    dev = gpu_forward(p.D, p.Q, p.w, "sum")
    D = t.from_numpy(p.D).pin_memory()
    Q = t.from_numpy(p.Q).pin_memory()
    w = t.from_numpy(p.w).pin_memory()
    host = domagg.forward_host(D, Q, w, "sum").numpy()
    assert np.array_equal(dev.view(np.uint32), host.view(np.uint32))
    pageable = domagg.forward_host(t.from_numpy(p.D), t.from_numpy(p.Q), t.from_numpy(p.w), "sum").numpy()
    assert np.array_equal(dev.view(np.uint32), pageable.view(np.uint32))


def test_invalid_arguments_are_rejected():
    h = domagg.handle(0)
    L = domagg.lib()
    st = L.domagg_forward(h, 5, None, 0, None, 0, 0, None, 1, 0, None, None)
    assert domagg.STATUS[st] == "UNSUPPORTED"
    st = L.domagg_forward(h, 0, None, 0, None, 0, 0, None, 1, 0, None, None)
    assert domagg.STATUS[st] == "INVALID_ARG"
    st = L.domagg_forward(h, 2, None, 5, None, 5, 0, None, 1, 0, None, None)
    assert domagg.STATUS[st] == "INVALID_ARG"
    st = L.domagg_forward(h, 2, None, 0, None, 0, 0, None, 0, 0, None, None)  # SUM of i32 weights
    assert domagg.STATUS[st] == "INVALID_ARG"
    st = L.domagg_forward(h, 2, None, 2**30, None, 2**30, 0, None, 1, 0, None, None)
    assert domagg.STATUS[st] == "UNSUPPORTED"
