"""The allocation-free forward entry point (domagg_forward_noalloc).

It serves callers that cannot allocate device memory; its scratch is one
static device array shared by every call.  These tests call it through the
C ABI and compare it with domagg_forward on two calls in a row (the second
call reuses the scratch the first one left behind).  The file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import assert_matches_oracle, to_dev, torch
from paper_2305_16751_gb300 import domagg, workloads

pytestmark = pytest.mark.gpu


def _noalloc(D, Q, w, op):
    t = torch()
    m = D.shape[1]
    out = t.empty(Q.shape[0], dtype=domagg.out_dtype(op, w), device=D.device)
    st = domagg.lib().domagg_forward_noalloc(
        m, ctypes.c_void_p(D.data_ptr()), D.shape[0], ctypes.c_void_p(Q.data_ptr()), Q.shape[0],
        domagg._coord_dtype(D), None if w is None else ctypes.c_void_p(w.data_ptr()), domagg._weight_dtype(w, op),
        domagg.OPS[op], ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(t.cuda.current_stream().cuda_stream))
    t.cuda.synchronize()
    return st, out


def _cases():
    rng = np.random.default_rng(31)
    p = workloads.tied_floats(n=12000)
    yield "m2 f32 sum", p.D, p.Q, p.w, "sum"
    D, Q, w = workloads.random_small(rng, 3, 6000, 5000, 3000, "i32", "i64")
    yield "m3 i64 sum", D, Q, w, "sum"
    D, Q, w = workloads.random_small(rng, 2, 20000, 15000, 40000, "f32", "i32")
    yield "m2 i32 max", D, Q, w, "max"


@pytest.mark.parametrize("case", range(3))
def test_noalloc_matches_forward_on_two_calls(case):
    name, D, Q, w, op = list(_cases())[case]
    Dd, Qd, wd = to_dev(D), to_dev(Q), to_dev(w)
    ref = domagg.forward(Dd, Qd, wd, op).cpu().numpy()
    for _ in range(2):
        st, out = _noalloc(Dd, Qd, wd, op)
        assert st == 0, (name, domagg.STATUS.get(st))
        got = out.cpu().numpy()
        if w.dtype == np.float32 and op == "sum":
            # float sums: both within the stated tolerance of the fp64 oracle
            assert_matches_oracle(got, D, Q, w, op)
        else:
            assert np.array_equal(got, ref), name


def test_noalloc_rejects_inputs_beyond_its_scratch():
    D = to_dev(np.zeros((40000, 2), np.int32))
    Q = to_dev(np.ones((40000, 2), np.int32))
    w = to_dev(np.ones(40000, np.int64))
    st, _ = _noalloc(D, Q, w, "sum")
    assert domagg.STATUS[st] == "UNSUPPORTED"


def test_noalloc_refuses_an_oversized_flat_map_then_works():
    """Under the point limit but with a flat map too large for the scratch
    (m = 3, 30000 points per side, a third of them on one first coordinate:
    the group holding them is too large for shared memory at every width,
    so no level is taken in groups and all 16 levels' records would go
    through the scratch): refused after the point phase, with `out`
    untouched; the next call on the same scratch is still correct."""
    rng = np.random.default_rng(32)
    D, Q, w = workloads.random_small(rng, 3, 30000, 30000, 1 << 20, "i32", "i64")
    D[:10000, 0] = 5
    Q[:10000, 0] = 5
    Dd, Qd, wd = to_dev(D), to_dev(Q), to_dev(w)
    t = torch()
    sentinel = t.full((Q.shape[0],), 12345, dtype=t.int64, device=Dd.device)
    st = domagg.lib().domagg_forward_noalloc(
        3, ctypes.c_void_p(Dd.data_ptr()), D.shape[0], ctypes.c_void_p(Qd.data_ptr()), Q.shape[0],
        domagg._coord_dtype(Dd), ctypes.c_void_p(wd.data_ptr()), domagg._weight_dtype(wd, "sum"),
        domagg.OPS["sum"], ctypes.c_void_p(sentinel.data_ptr()), ctypes.c_void_p(t.cuda.current_stream().cuda_stream))
    t.cuda.synchronize()
    assert domagg.STATUS[st] == "UNSUPPORTED"
    assert bool((sentinel == 12345).all())
    name, D2, Q2, w2, op = list(_cases())[1]
    D2d, Q2d, w2d = to_dev(D2), to_dev(Q2), to_dev(w2)
    st, out = _noalloc(D2d, Q2d, w2d, op)
    assert st == 0
    assert np.array_equal(out.cpu().numpy(), domagg.forward(D2d, Q2d, w2d, op).cpu().numpy())


def test_noalloc_m3_groups_fit_the_scratch():
    """m = 3 with 30000 spread points per side: the first-rank levels below
    the groups are formed in shared memory, the three above go through the
    scratch; two calls in a row equal domagg_forward."""
    rng = np.random.default_rng(33)
    D, Q, w = workloads.random_small(rng, 3, 30000, 30000, 1 << 20, "i32", "i64")
    Dd, Qd, wd = to_dev(D), to_dev(Q), to_dev(w)
    ref = domagg.forward(Dd, Qd, wd, "sum").cpu().numpy()
    for _ in range(2):
        st, out = _noalloc(Dd, Qd, wd, "sum")
        assert st == 0, domagg.STATUS.get(st)
        assert np.array_equal(out.cpu().numpy(), ref)
