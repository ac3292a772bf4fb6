"""Backward (reverse dominance) and batched launches on the GPU, against the
oracle's transposed brute force and against single-instance calls."""
import numpy as np
import pytest

import oracle
from gpu_helpers import F32_TOL, assert_matches_oracle, gpu_forward, to_dev, torch
from paper_2305_16751_gb300 import domagg, workloads

pytestmark = pytest.mark.gpu


def _check_grad(got, want, S):
    err = np.abs(got.astype(np.float64) - want)
    bad = np.nonzero(err > F32_TOL * S)[0]
    assert bad.size == 0, f"{bad.size} out of tolerance, e.g. {bad[:5]}"


@pytest.mark.parametrize("m,dt", [(1, "f32"), (2, "f32"), (2, "i32"), (3, "i32"), (3, "f32")])
def test_backward_matches_transposed_brute_force(m, dt):
    rng = np.random.default_rng(50 + m)
    D, Q, _ = workloads.random_small(rng, m, 7000, 9000, 60, dt, "f32")
    g = rng.standard_normal(9000).astype(np.float32)
    got = domagg.backward(to_dev(D), to_dev(Q), to_dev(g)).cpu().numpy()
    want, S = oracle.brute_transpose(D, Q, g)
    _check_grad(got, want, S)


def test_autograd_function_fd_workload():
    """loss = sum_q c_q out_q on the autograd workload shape (small n):
    w.grad equals the transposed sum; D and Q get no gradient."""
    t = torch()
    p = workloads.autograd_floats(n=20000)
    D, Q = to_dev(p.D), to_dev(p.Q)
    w = to_dev(p.w).requires_grad_(True)
    c = to_dev(p.extra["c"])
    out = domagg.dominance_sum(D, Q, w)
    (out * c).sum().backward()
    want, S = oracle.brute_transpose(p.D, p.Q, p.extra["c"])
    _check_grad(w.grad.cpu().numpy(), want, S)
    assert_matches_oracle(out.detach().cpu().numpy(), p.D, p.Q, p.w, "sum")
    assert D.grad is None and Q.grad is None


def test_autograd_at_512_matches_oracle_finite_differences():
    """The gradient through autograd equals central finite differences of the
    fp64 oracle loss at |D| = |Q| = 512 (the loss is linear in w)."""
    p = workloads.autograd_floats(n=512)
    rng = np.random.default_rng(0)
    w0 = (rng.integers(-2048, 2048, size=512) * 2.0**-10).astype(np.float32)
    c = p.extra["c"]
    w = to_dev(w0).requires_grad_(True)
    (domagg.dominance_sum(to_dev(p.D), to_dev(p.Q), w) * to_dev(c)).sum().backward()
    h = np.float32(2.0**-10)

    def L(wv):
        return float(np.dot(c.astype(np.float64), oracle.brute(p.D, p.Q, wv, "sum")[0]))

    fd = np.empty(512)
    for d in range(512):
        wp, wm = w0.copy(), w0.copy()
        wp[d] += h
        wm[d] -= h
        fd[d] = (L(wp) - L(wm)) / (2 * float(h))
    S = oracle.brute_transpose(p.D, p.Q, c)[1]
    _check_grad(w.grad.cpu().numpy(), fd, S)


@pytest.mark.parametrize("op,wt", [("sum", "f32"), ("sum", "i64"), ("max", "i32"), ("count", "i64"), ("min", "f32")])
def test_batch_equals_single_calls(op, wt):
    rng = np.random.default_rng(77)
    probs = []
    for i in range(40):
        m = int(rng.integers(1, 4))
        nD, nQ = int(rng.integers(0, 3000)), int(rng.integers(0, 3000))
        if i % 13 == 5:
            nD = 0
        D, Q, w = workloads.random_small(rng, m, nD, nQ, int(rng.integers(2, 500)), "i32", wt)
        probs.append((D, Q, w))
    outs = domagg.batch([(to_dev(D), to_dev(Q), to_dev(w)) for D, Q, w in probs], op)
    torch().cuda.synchronize()
    for (D, Q, w), o in zip(probs, outs):
        o = o.cpu().numpy()
        single = gpu_forward(D, Q, w if op != "count" else None, op)
        assert np.array_equal(o.view(np.uint8), single.view(np.uint8))
        assert_matches_oracle(o, D, Q, w if op != "count" else None, op)


def test_batch_workload_shape_small():
    """The batch workload (uniform int32 coordinates in [0, 2^31), float32
    weights) at reduced instance count and sizes."""
    probs = workloads.batch_instances(k=64, lo=64, hi=4096)
    outs = domagg.batch([(to_dev(p.D), to_dev(p.Q), to_dev(p.w)) for p in probs], "sum")
    torch().cuda.synchronize()
    for p, o in zip(probs, outs):
        assert_matches_oracle(o.cpu().numpy(), p.D, p.Q, p.w, "sum")


def test_batch_split_into_record_chunks():
    """A handle whose workspace cap is small processes a batch in several
    record chunks (a synchronisation between them); results equal the
    single calls."""
    import ctypes
    t = torch()
    rng = np.random.default_rng(5)
    probs = []
    for i in range(12):
        m = 2 + (i % 2)
        D, Q, w = workloads.random_small(rng, m, 3000 + 100 * i, 2500, 2000, "i32", "i64")
        probs.append((D, Q, w))
    h = domagg.domagg_create(0, 64 << 20)
    try:
        arr = (domagg.domagg_instance * len(probs))()
        keep, outs = [], []
        for i, (D, Q, w) in enumerate(probs):
            Dd, Qd, wd = to_dev(D), to_dev(Q), to_dev(w)
            o = t.empty(Q.shape[0], dtype=t.int64, device="cuda")
            keep += [Dd, Qd, wd]
            outs.append(o)
            arr[i] = domagg.domagg_instance(D.shape[1], D.shape[0], Q.shape[0], Dd.data_ptr(), Qd.data_ptr(),
                                            wd.data_ptr(), o.data_ptr())
        domagg.domagg_batch(h, len(probs), arr, domagg.DTYPES["i32"], domagg.DTYPES["i64"], domagg.OPS["sum"],
                            ctypes.c_void_p(t.cuda.current_stream().cuda_stream))
        t.cuda.synchronize()
        for (D, Q, w), o in zip(probs, outs):
            assert np.array_equal(o.cpu().numpy(), gpu_forward(D, Q, w, "sum"))
    finally:
        domagg.domagg_destroy(h)


def test_batch_full_recipe_sampled():
    """The full batch workload (4096 instances, 3.0e8 points) in one
    domagg_batch call, as the bench times it; 24 sampled instances, 32
    sampled queries each, against the oracle."""
    probs = workloads.batch_instances()
    dev = [(to_dev(p.D), to_dev(p.Q), to_dev(p.w)) for p in probs]
    outs = domagg.batch(dev, "sum")
    torch().cuda.synchronize()
    rng = np.random.default_rng(11)
    for i in np.sort(rng.choice(len(probs), 24, replace=False)):
        p = probs[i]
        qi = np.sort(rng.choice(p.Q.shape[0], 32, replace=False))
        assert_matches_oracle(outs[i].cpu().numpy(), p.D, p.Q, p.w, "sum", qidx=qi)
