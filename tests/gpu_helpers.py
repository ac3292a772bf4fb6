"""Shared helpers of the GPU parity tests: run the CUDA path through the
C ABI and compare with the CPU oracle."""
import numpy as np

import oracle

F32_TOL = 4.0 * 2.0**-24  # |gpu - fp64| <= F32_TOL * sum |w| over the dominated set


def torch():
    import torch as t
    return t


def to_dev(a):
    t = torch()
    return None if a is None else t.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_forward(D, Q, w, op):
    from paper_2305_16751_gb300 import domagg
    out = domagg.forward(to_dev(D), to_dev(Q), to_dev(w), op)
    torch().cuda.synchronize()
    return out.cpu().numpy()


def assert_matches_oracle(got, D, Q, w, op, want=None, S=None, qidx=None):
    """Bit-exact for integer results, F32_TOL * S for float32 sums, and exact
    for float32 max."""
    if want is None:
        Dq = Q if qidx is None else Q[qidx]
        want, S = oracle.brute(D, Dq, w, op)
    if qidx is not None:
        got = got[qidx]
    if op == "sum" and w is not None and w.dtype == np.float32:
        err = np.abs(got.astype(np.float64) - want)
        bound = F32_TOL * S
        bad = np.nonzero(err > bound)[0]
        assert bad.size == 0, f"{bad.size} queries out of tolerance, first {bad[:5]}: got {got[bad[:5]]} want {want[bad[:5]]}"
    elif op in ("max", "min") and w is not None and w.dtype == np.float32:
        assert np.array_equal(got.astype(np.float64), want)
    else:
        assert np.array_equal(got.astype(np.int64), want.astype(np.int64)), \
            f"first mismatch at {np.nonzero(got.astype(np.int64) != want)[0][:5]}"


_FULL_CACHE = {}


def full_size_m2_oracle(weights: str, op: str):
    """The full-size m = 2 workload (|D| = |Q| = 2^24, float32 coordinates
    with 25% quantised) and its oracle result on EVERY query, by the
    O(n log n) sweep (pinned to brute force on the CPU); cached per process so
    several GPU variants share one oracle run.  Returns (problem, want, S)."""
    from paper_2305_16751_gb300 import workloads
    key = (weights, op)
    if key not in _FULL_CACHE:
        p = workloads.tied_floats(weights=weights)
        want, S = oracle.sweep2(p.D, p.Q, p.w, op)
        _FULL_CACHE[key] = (p, want, S)
    return _FULL_CACHE[key]
