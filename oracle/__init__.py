"""CPU oracle for aggregation over dominated points (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library never loads it, and it imports nothing from the product
package.  See ``domagg_oracle.c`` for what each routine computes and which
passage of the paper it follows.

Every routine here calls the C oracle through ctypes; the numpy code around
the calls only checks shapes, converts types and allocates outputs.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build_oracle

_HERE = os.path.dirname(os.path.abspath(__file__))

# Enumerations of the C oracle (its own numbering).
COORD = {"i32": 0, "f32": 2}
WEIGHT = {"i32": 0, "i64": 1, "f32": 2}
OPS = {"sum": 0, "max": 1, "count": 2, "min": 3}

_libs: dict[int, ctypes.CDLL] = {}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle returned status {code}")
        self.code = code


def _lib(plant: int = 0) -> ctypes.CDLL:
    if plant not in _libs:
        path = build_oracle(plant)
        lib = ctypes.CDLL(path)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.oracle_brute.argtypes = [i32, vp, i64, vp, i64, i32, vp, i32, i32, vp, vp, i32]
        lib.oracle_brute.restype = i32
        lib.oracle_brute_ns.argtypes = [i32, vp, i64, vp, i64, i32, vp, i32, i32, ctypes.c_uint32, vp, vp, i32]
        lib.oracle_brute_ns.restype = i32
        lib.oracle_brute_transpose.argtypes = [i32, vp, i64, vp, i64, i32, vp, vp, vp, i32]
        lib.oracle_brute_transpose.restype = i32
        lib.oracle_sortscan.argtypes = [i32, vp, i64, vp, i64, i32, vp, i32, i32, vp, vp]
        lib.oracle_sortscan.restype = i32
        lib.oracle_sscan_i64.argtypes = [vp, vp, i64, vp]
        lib.oracle_sscan_i64.restype = None
        lib.oracle_prefix_set.argtypes = [ctypes.c_uint64, i32, i32, vp, vp]
        lib.oracle_prefix_set.restype = i32
        lib.oracle_sweep2.argtypes = [vp, i64, vp, i64, i32, vp, i32, i32, ctypes.c_uint32, vp, vp]
        lib.oracle_sweep2.restype = i32
        lib.oracle_sweep2_transpose.argtypes = [vp, i64, vp, i64, i32, vp, ctypes.c_uint32, vp, vp]
        lib.oracle_sweep2_transpose.restype = i32
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = i32
        _libs[plant] = lib
    return _libs[plant]


def _ptr(a: np.ndarray | None):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _coords(x: np.ndarray, m: int) -> tuple[np.ndarray, int]:
    x = np.ascontiguousarray(x)
    if x.ndim != 2 or x.shape[1] != m:
        raise ValueError(f"coordinates must be [n, {m}]")
    if x.dtype == np.int32:
        return x, COORD["i32"]
    if x.dtype == np.float32:
        return x, COORD["f32"]
    raise TypeError(f"coordinates must be int32 or float32, got {x.dtype}")


def _weights(w: np.ndarray | None, nD: int, op: str) -> tuple[np.ndarray | None, int]:
    if op == "count":
        return None, WEIGHT["i64"]
    w = np.ascontiguousarray(w)
    if w.shape != (nD,):
        raise ValueError("weights must be [nD]")
    key = {np.dtype(np.int32): "i32", np.dtype(np.int64): "i64", np.dtype(np.float32): "f32"}.get(w.dtype)
    if key is None:
        raise TypeError(f"weights must be int32, int64 or float32, got {w.dtype}")
    return w, WEIGHT[key]


def _out_array(n: int, wt: int, op: str) -> np.ndarray:
    is_float = op != "count" and wt == WEIGHT["f32"]
    return np.empty(n, dtype=np.float64 if is_float else np.int64)


def brute(D, Q, w, op: str, threads: int = 0, plant: int = 0, nonstrict: int = 0):
    """Definition of Sec. 1.2 by brute force.  Returns (out, S) with
    S[q] = sum of |w(d)| over the dominated set (float64).  Bit i of
    `nonstrict` compares coordinate i as d_i <= q_i."""
    m = D.shape[1]
    D, ct = _coords(D, m)
    Q, ct2 = _coords(Q, m)
    if ct != ct2:
        raise TypeError("D and Q must have the same dtype")
    w, wt = _weights(w, D.shape[0], op)
    out = _out_array(Q.shape[0], wt, op)
    S = np.empty(Q.shape[0], dtype=np.float64)
    st = _lib(plant).oracle_brute_ns(m, _ptr(D), D.shape[0], _ptr(Q), Q.shape[0], ct, _ptr(w), wt,
                                     OPS[op], nonstrict, _ptr(out), _ptr(S), threads)
    if st:
        raise OracleError(st)
    return out, S


def brute_transpose(D, Q, g, threads: int = 0, plant: int = 0):
    """grad[d] = sum of g[q] over queries q that dominate d (float64), and
    S[d] = sum of |g[q]| over the same set."""
    m = D.shape[1]
    D, ct = _coords(D, m)
    Q, _ = _coords(Q, m)
    g = np.ascontiguousarray(g, dtype=np.float32)
    grad = np.empty(D.shape[0], dtype=np.float64)
    S = np.empty(D.shape[0], dtype=np.float64)
    st = _lib(plant).oracle_brute_transpose(m, _ptr(D), D.shape[0], _ptr(Q), Q.shape[0], ct,
                                            _ptr(g), _ptr(grad), _ptr(S), threads)
    if st:
        raise OracleError(st)
    return grad, S


def sweep2(D, Q, w, op: str, nonstrict: int = 0, plant: int = 0):
    """m = 2 by a sweep over the last coordinate with a Fenwick tree over the
    first coordinate's ranks (O(n log n); not the paper's algorithm, pinned to
    brute force by the tests).  Returns (out, S) like brute()."""
    D, ct = _coords(D, 2)
    Q, ct2 = _coords(Q, 2)
    if ct != ct2:
        raise TypeError("D and Q must have the same dtype")
    w, wt = _weights(w, D.shape[0], op)
    out = _out_array(Q.shape[0], wt, op)
    S = np.empty(Q.shape[0], dtype=np.float64)
    st = _lib(plant).oracle_sweep2(_ptr(D), D.shape[0], _ptr(Q), Q.shape[0], ct, _ptr(w), wt, OPS[op],
                                   nonstrict, _ptr(out), _ptr(S))
    if st:
        raise OracleError(st)
    return out, S


def sweep2_transpose(D, Q, g, nonstrict: int = 0, plant: int = 0):
    """The adjoint for m = 2 by the sweep: grad[d] = sum of g[q] over queries q
    that dominate d, and S[d] = sum of |g[q]| over the same set."""
    D, ct = _coords(D, 2)
    Q, _ = _coords(Q, 2)
    g = np.ascontiguousarray(g, dtype=np.float32)
    grad = np.empty(D.shape[0], dtype=np.float64)
    S = np.empty(D.shape[0], dtype=np.float64)
    st = _lib(plant).oracle_sweep2_transpose(_ptr(D), D.shape[0], _ptr(Q), Q.shape[0], ct, _ptr(g), nonstrict,
                                             _ptr(grad), _ptr(S))
    if st:
        raise OracleError(st)
    return grad, S


def sortscan(D, Q, w, op: str, plant: int = 0):
    """The paper's algorithm (Sec. 4 with Sec. 5).  Returns (out, T) with T
    the number of records produced by the flat map."""
    m = D.shape[1]
    D, ct = _coords(D, m)
    Q, _ = _coords(Q, m)
    w, wt = _weights(w, D.shape[0], op)
    out = _out_array(Q.shape[0], wt, op)
    T = ctypes.c_int64(0)
    st = _lib(plant).oracle_sortscan(m, _ptr(D), D.shape[0], _ptr(Q), Q.shape[0], ct, _ptr(w), wt,
                                     OPS[op], _ptr(out), ctypes.byref(T))
    if st:
        raise OracleError(st)
    return out, int(T.value)


def record_count(D, Q, plant: int = 0) -> int:
    """Number of records of the flat map (Sec. 5), computed by the oracle."""
    m = D.shape[1]
    D, ct = _coords(D, m)
    Q, _ = _coords(Q, m)
    T = ctypes.c_int64(0)
    st = _lib(plant).oracle_sortscan(m, _ptr(D), D.shape[0], _ptr(Q), Q.shape[0], ct, None,
                                     WEIGHT["i64"], OPS["count"], None, ctypes.byref(T))
    if st:
        raise OracleError(st)
    return int(T.value)


def sscan_i64(a, t) -> np.ndarray:
    """Segmented scan with + (Sec. 2.2), by its definition."""
    a = np.ascontiguousarray(a, dtype=np.int64)
    t = np.ascontiguousarray(t, dtype=np.int64)
    out = np.empty_like(a)
    _lib().oracle_sscan_i64(_ptr(a), _ptr(t), a.shape[0], _ptr(out))
    return out


def prefix_set(x: int, b: int, which: int) -> list[str]:
    """P0(x) (which=0) or P1(x) (which=1) of Sec. 3 as bitstrings."""
    lens = np.zeros(64, dtype=np.int32)
    vals = np.zeros(64, dtype=np.uint64)
    n = _lib().oracle_prefix_set(x, b, which, _ptr(lens), _ptr(vals))
    out = []
    for k in range(n):
        L = int(lens[k])
        out.append(format(int(vals[k]), f"0{L}b") if L else "")
    return out


def max_threads() -> int:
    return int(_lib().oracle_max_threads())
