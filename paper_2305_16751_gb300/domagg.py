"""Python binding of the domagg C ABI (include/domagg.h).

The functions named ``domagg_*`` mirror the C entry points one to one and
only marshal arguments through ctypes.  The torch-level helpers below them
(``forward``, ``backward``, ``DominanceSum``, ``batch``) allocate output
tensors with torch and pass raw device pointers and the current CUDA stream;
every step of the computation runs in the library's CUDA kernels.  There is
no fallback: if the library is not built, or no GPU is present, the calls
raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB, LIB_CHECKED

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OOM", 4: "CUDA", 5: "TIMEOUT", 6: "NAN", 7: "BOUNDS"}
OPS = {"sum": 0, "max": 1, "count": 2, "min": 3}
DTYPES = {"i32": 0, "i64": 1, "f32": 2}
TIMING_KINDS = 20


class DomaggError(RuntimeError):
    def __init__(self, status: int, message: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"domagg error {self.name}: {message}")


class domagg_instance(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("nD", ctypes.c_int64), ("nQ", ctypes.c_int64),
                ("d_coords", ctypes.c_void_p), ("q_coords", ctypes.c_void_p),
                ("d_weights", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class domagg_stats(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_records", ctypes.c_int64),
                ("n_query_records", ctypes.c_int64), ("m", ctypes.c_int32),
                ("rank_bits", ctypes.c_int32 * 3), ("distinct", ctypes.c_int64 * 3),
                ("record_key_bits", ctypes.c_int32), ("record_passes", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_int64), ("n_records_shared", ctypes.c_int64)]


class domagg_timing(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int32 * TIMING_KINDS), ("ms", ctypes.c_double * TIMING_KINDS),
                ("bytes", ctypes.c_double * TIMING_KINDS)]


# Every symbol the header declares, with its ctypes signature.
_vp, _i64, _int, _sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
SIGNATURES = {
    "domagg_create": ([ctypes.POINTER(_vp), _int, _sz], _int),
    "domagg_destroy": ([_vp], _int),
    "domagg_forward": ([_vp, _int, _vp, _i64, _vp, _i64, _int, _vp, _int, _int, _vp, _vp], _int),
    "domagg_forward_ex": ([_vp, _int, _vp, _i64, _vp, _i64, _int, _vp, _int, _int, ctypes.c_uint32, _int, _vp, _vp],
                          _int),
    "domagg_forward_host": ([_vp, _int, _vp, _i64, _vp, _i64, _int, _vp, _int, _int, _vp, _vp], _int),
    "domagg_forward_shard": ([_vp, _int, _int, _int, _vp, _i64, _vp, _i64, _int, _vp, _int, _int, _vp, _vp, _vp],
                             _int),
    "domagg_combine": ([_vp, _int, _int, _int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i64, _vp, _vp], _int),
    "domagg_ecdf_distance": ([_vp, _vp, _vp, _i64, _i64, _i64, _vp, _vp], _int),
    "domagg_backward": ([_vp, _int, _vp, _i64, _vp, _i64, _int, _vp, _vp, _vp], _int),
    "domagg_backward_ex": ([_vp, _int, _vp, _i64, _vp, _i64, _int, _vp, _vp, ctypes.c_uint32, _int, _vp], _int),
    "domagg_batch": ([_vp, _int, ctypes.POINTER(domagg_instance), _int, _int, _int, _vp], _int),
    "domagg_batch_plan": ([ctypes.POINTER(_vp), _int, _int, ctypes.POINTER(domagg_instance), _int, _int, _int,
                           ctypes.c_double, _vp], _int),
    "domagg_plan_run": ([_vp, _vp], _int),
    "domagg_plan_status": ([_vp, _vp], _int),
    "domagg_plan_autotune": ([_vp, _vp, ctypes.POINTER(ctypes.c_double)], _int),
    "domagg_plan_last_error": ([_vp], ctypes.c_char_p),
    "domagg_plan_workspace_bytes": ([_vp], _i64),
    "domagg_plan_destroy": ([_vp], _int),
    "domagg_sync_status": ([_vp, _vp], _int),
    "domagg_selftest_timeout": ([_vp, _int, _vp], _int),
    "domagg_last_error": ([_vp], ctypes.c_char_p),
    "domagg_get_stats": ([_vp, ctypes.POINTER(domagg_stats)], _int),
    "domagg_timing_enable": ([_vp, _int], _int),
    "domagg_timing_read": ([_vp, ctypes.POINTER(domagg_timing)], _int),
    "domagg_set_tuning": ([_vp, ctypes.c_char_p, _int], _int),
    "domagg_timing_kind_name": ([_int], ctypes.c_char_p),
    "domagg_version": ([], ctypes.c_char_p),
    "domagg_forward_noalloc": ([_int, _vp, _i64, _vp, _i64, _int, _vp, _int, _int, _vp, _vp], _int),
}

_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Loads the in-tree library; raises if it has not been built.  With the
    environment variable DOMAGG_CHECKED=1 the checked build is loaded instead
    (kernels test every computed index; a miss returns DOMAGG_ERR_BOUNDS)."""
    global _lib
    with _lock:
        if _lib is None:
            path = LIB_CHECKED if os.environ.get("DOMAGG_CHECKED") == "1" else LIB
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
            L = ctypes.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(h, st: int):
    if st != 0:
        msg = lib().domagg_last_error(h).decode() if h else ""
        raise DomaggError(st, msg)


# --- the C entry points, one to one -----------------------------------------

def domagg_create(device: int = 0, max_workspace_bytes: int = 0):
    h = ctypes.c_void_p()
    _check(None, lib().domagg_create(ctypes.byref(h), device, max_workspace_bytes))
    return h


def domagg_destroy(h):
    _check(None, lib().domagg_destroy(h))


def domagg_forward(h, m, d_coords, nD, q_coords, nQ, coord_dtype, d_weights, weight_dtype, op, out, stream):
    _check(h, lib().domagg_forward(h, m, d_coords, nD, q_coords, nQ, coord_dtype, d_weights, weight_dtype, op,
                                   out, stream))


def domagg_forward_ex(h, m, d_coords, nD, q_coords, nQ, coord_dtype, d_weights, weight_dtype, op, nonstrict_mask,
                      variant, out, stream):
    _check(h, lib().domagg_forward_ex(h, m, d_coords, nD, q_coords, nQ, coord_dtype, d_weights, weight_dtype, op,
                                      nonstrict_mask, variant, out, stream))


def domagg_forward_host(h, m, d_coords, nD, q_coords, nQ, coord_dtype, d_weights, weight_dtype, op, out, stream):
    _check(h, lib().domagg_forward_host(h, m, d_coords, nD, q_coords, nQ, coord_dtype, d_weights, weight_dtype,
                                        op, out, stream))


def domagg_backward(h, m, d_coords, nD, q_coords, nQ, coord_dtype, grad_out, grad_w, stream):
    _check(h, lib().domagg_backward(h, m, d_coords, nD, q_coords, nQ, coord_dtype, grad_out, grad_w, stream))


def domagg_batch(h, k, inst_array, coord_dtype, weight_dtype, op, stream):
    _check(h, lib().domagg_batch(h, k, inst_array, coord_dtype, weight_dtype, op, stream))


def domagg_sync_status(h, stream):
    _check(h, lib().domagg_sync_status(h, stream))


def _check_plan(p, st: int):
    if st != 0:
        raise DomaggError(st, lib().domagg_plan_last_error(p).decode())


def domagg_batch_plan(device, k, inst_array, coord_dtype, weight_dtype, op, headroom, stream):
    p = ctypes.c_void_p()
    st = lib().domagg_batch_plan(ctypes.byref(p), device, k, inst_array, coord_dtype, weight_dtype, op, headroom,
                                 stream)
    _check_plan(None, st)
    return p


def domagg_plan_run(p, stream):
    _check_plan(p, lib().domagg_plan_run(p, stream))


def domagg_plan_status(p, stream):
    _check_plan(p, lib().domagg_plan_status(p, stream))


def domagg_plan_autotune(p, stream) -> float:
    ms = ctypes.c_double()
    _check_plan(p, lib().domagg_plan_autotune(p, stream, ctypes.byref(ms)))
    return ms.value


def domagg_plan_workspace_bytes(p) -> int:
    return int(lib().domagg_plan_workspace_bytes(p))


def domagg_plan_destroy(p):
    _check_plan(None, lib().domagg_plan_destroy(p))


def domagg_get_stats(h) -> dict:
    s = domagg_stats()
    _check(h, lib().domagg_get_stats(h, ctypes.byref(s)))
    return {"n_points": s.n_points, "n_records": s.n_records, "n_query_records": s.n_query_records,
            "m": s.m, "rank_bits": list(s.rank_bits), "distinct": list(s.distinct),
            "record_key_bits": s.record_key_bits, "record_passes": s.record_passes,
            "workspace_bytes": s.workspace_bytes, "n_records_shared": s.n_records_shared}


def domagg_set_tuning(h, name: str, value: int):
    """A tuning knob of the handle (see include/domagg.h): "group_bits",
    "top_bits", "rank_windows", "ranges_per_cta" or "blocks_per_sm"."""
    _check(h, lib().domagg_set_tuning(h, name.encode(), int(value)))


def domagg_timing_enable(h, enable: bool):
    _check(h, lib().domagg_timing_enable(h, 1 if enable else 0))


def domagg_timing_read(h) -> dict:
    t = domagg_timing()
    _check(h, lib().domagg_timing_read(h, ctypes.byref(t)))
    out = {}
    for k in range(TIMING_KINDS):
        name = lib().domagg_timing_kind_name(k).decode()
        if name and t.launches[k]:
            out[name] = {"launches": t.launches[k], "ms": t.ms[k], "bytes": t.bytes[k]}
    return out


def domagg_version() -> str:
    return lib().domagg_version().decode()


# --- torch-level helpers -----------------------------------------------------

_handles: dict[int, ctypes.c_void_p] = {}


def handle(device: int = 0):
    """One library handle per device, created on first use."""
    with _lock:
        h = _handles.get(device)
    if h is None:
        h = domagg_create(device)
        with _lock:
            _handles[device] = h
    return h


def _torch():
    import torch
    return torch


def _coord_dtype(t) -> int:
    torch = _torch()
    if t.dtype == torch.int32:
        return DTYPES["i32"]
    if t.dtype == torch.float32:
        return DTYPES["f32"]
    raise TypeError("coordinates must be int32 or float32")


def _weight_dtype(w, op: str) -> int:
    torch = _torch()
    if op == "count":
        return DTYPES["i64"]
    return {torch.int32: DTYPES["i32"], torch.int64: DTYPES["i64"], torch.float32: DTYPES["f32"]}[w.dtype]


def out_dtype(op: str, w):
    torch = _torch()
    if op == "count":
        return torch.int64
    return w.dtype


def _stream(dev):
    return ctypes.c_void_p(_torch().cuda.current_stream(dev).cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else None


VARIANTS = {"improved": 0, "basic": 1, "wavelet": 2}


def forward(D, Q, w=None, op: str = "sum", out=None, nonstrict: int = 0, variant: str = "improved"):
    """out[q] = F over w(d) for d < q (strict), computed on D's GPU.  Bit i
    of `nonstrict` compares coordinate i as d_i <= q_i; variant "basic" runs
    the unimproved algorithm of Sec. 4 (m <= 3), variant "wavelet" the
    level-wise formulation of the first coordinate (m <= 2, no records)."""
    torch = _torch()
    if D.device.type != "cuda":
        raise ValueError("forward expects CUDA tensors (use forward_host for host buffers)")
    D, Q = D.contiguous(), Q.contiguous()
    m = D.shape[1]
    if Q.shape[1] != m or Q.dtype != D.dtype:
        raise ValueError("D and Q must have the same width and dtype")
    w = None if op == "count" else w.contiguous()
    if out is None:
        out = torch.empty(Q.shape[0], dtype=out_dtype(op, w), device=D.device)
    dev = D.device.index or 0
    if nonstrict or variant != "improved":
        domagg_forward_ex(handle(dev), m, _ptr(D), D.shape[0], _ptr(Q), Q.shape[0], _coord_dtype(D), _ptr(w),
                          _weight_dtype(w, op), OPS[op], nonstrict, VARIANTS[variant], _ptr(out), _stream(D.device))
    else:
        domagg_forward(handle(dev), m, _ptr(D), D.shape[0], _ptr(Q), Q.shape[0], _coord_dtype(D), _ptr(w),
                       _weight_dtype(w, op), OPS[op], _ptr(out), _stream(D.device))
    return out


def forward_shard(D, Q, w, op: str, shard: int, nshards: int):
    """Shard `shard` of `nshards` of forward(D, Q, w, op) (domagg_forward_shard):
    F over the shard's part of the flat map.  Returns (out, out_lo); out_lo
    holds the low halves of the float-float partials of a float32 sum (None
    for other ops)."""
    torch = _torch()
    D, Q = D.contiguous(), Q.contiguous()
    w = None if op == "count" else w.contiguous()
    out = torch.empty(Q.shape[0], dtype=out_dtype(op, w), device=D.device)
    out_lo = torch.empty(Q.shape[0], dtype=torch.float32, device=D.device) \
        if (op == "sum" and w is not None and w.dtype == torch.float32) else None
    dev = D.device.index or 0
    _check(handle(dev), lib().domagg_forward_shard(
        handle(dev), shard, nshards, D.shape[1], _ptr(D), D.shape[0], _ptr(Q), Q.shape[0], _coord_dtype(D), _ptr(w),
        _weight_dtype(w, op), OPS[op], _ptr(out), _ptr(out_lo), _stream(D.device)))
    return out, out_lo


def combine(parts, parts_lo, op: str, weight_dtype=None, out=None):
    """F over the shards' outputs (domagg_combine): parts are the `out`
    tensors of forward_shard, parts_lo their `out_lo` (or None)."""
    torch = _torch()
    n = len(parts)
    dev = parts[0].device
    if out is None:
        out = torch.empty_like(parts[0])
    wd = {None: 1, torch.int32: 0, torch.int64: 1, torch.float32: 2}[weight_dtype if op != "count" else None]
    P = (_vp * n)(*[p.data_ptr() for p in parts])
    lo = (_vp * n)(*[x.data_ptr() for x in parts_lo]) if parts_lo is not None and parts_lo[0] is not None else None
    _check(handle(dev.index or 0), lib().domagg_combine(handle(dev.index or 0), OPS[op], wd, n, P, lo,
                                                        parts[0].shape[0], _ptr(out), _stream(dev)))
    return out


def ks_statistic(X, Y) -> float:
    """Two-sample statistic max over z in X u Y of |F_X(z) - F_Y(z)|, with F
    the empirical CDF (the fraction of a sample <= z in every coordinate):
    two dominance counts with every coordinate non-strict and their largest
    difference (domagg_ecdf_distance), on the GPU."""
    torch = _torch()
    Z = torch.cat([X, Y]).contiguous()
    full = (1 << X.shape[1]) - 1
    cx = forward(X, Z, None, "count", nonstrict=full)
    cy = forward(Y, Z, None, "count", nonstrict=full)
    out = torch.empty(1, dtype=torch.float64, device=Z.device)
    h = handle(Z.device.index or 0)
    _check(h, lib().domagg_ecdf_distance(h, _ptr(cx), _ptr(cy), Z.shape[0], X.shape[0], Y.shape[0], _ptr(out),
                                         _stream(Z.device)))
    return float(out.item())


def forward_host(D, Q, w=None, op: str = "sum", device: int = 0):
    """Same as forward, from host (CPU) tensors: the library copies the inputs
    to the GPU, runs, copies the result back and synchronises."""
    torch = _torch()
    D, Q = D.contiguous(), Q.contiguous()
    w = None if op == "count" else w.contiguous()
    out = torch.empty(Q.shape[0], dtype=out_dtype(op, w), pin_memory=D.is_pinned())
    domagg_forward_host(handle(device), D.shape[1], _ptr(D), D.shape[0], _ptr(Q), Q.shape[0], _coord_dtype(D),
                        _ptr(w), _weight_dtype(w, op), OPS[op], _ptr(out),
                        _stream(torch.device("cuda", device)))
    return out


def backward(D, Q, grad_out, nonstrict: int = 0, variant: str = "improved"):
    """grad_w[d] = sum of grad_out[q] over queries q with d < q (bit i of
    `nonstrict`: d_i <= q_i); variant "wavelet" (m <= 2) uses the level-wise
    formulation."""
    torch = _torch()
    D, Q = D.contiguous(), Q.contiguous()
    g = grad_out.contiguous().to(torch.float32)
    grad_w = torch.empty(D.shape[0], dtype=torch.float32, device=D.device)
    dev = D.device.index or 0
    if nonstrict or variant != "improved":
        _check(handle(dev), lib().domagg_backward_ex(handle(dev), D.shape[1], _ptr(D), D.shape[0], _ptr(Q),
                                                     Q.shape[0], _coord_dtype(D), _ptr(g), _ptr(grad_w),
                                                     nonstrict, VARIANTS[variant], _stream(D.device)))
    else:
        domagg_backward(handle(dev), D.shape[1], _ptr(D), D.shape[0], _ptr(Q), Q.shape[0], _coord_dtype(D),
                        _ptr(g), _ptr(grad_w), _stream(D.device))
    return grad_w


def _autograd_function():
    torch = _torch()

    class DominanceSum(torch.autograd.Function):
        """out = dominance sum of float32 weights; differentiable in w only
        (coordinates are piecewise constant: their gradient is None)."""

        @staticmethod
        def forward(ctx, D, Q, w, nonstrict=0, variant="improved"):
            ctx.save_for_backward(D, Q)
            ctx.nonstrict = nonstrict
            ctx.variant = variant
            return forward(D, Q, w, "sum", nonstrict=nonstrict, variant=variant)

        @staticmethod
        def backward(ctx, grad_out):
            D, Q = ctx.saved_tensors
            return None, None, backward(D, Q, grad_out, ctx.nonstrict, ctx.variant), None, None

    return DominanceSum


_DominanceSum = None


def dominance_sum(D, Q, w, nonstrict: int = 0, variant: str = "improved"):
    """Autograd-enabled float32 dominance sum (backward recomputes the
    records); bit i of `nonstrict` compares coordinate i as d_i <= q_i."""
    global _DominanceSum
    if _DominanceSum is None:
        _DominanceSum = _autograd_function()
    return _DominanceSum.apply(D, Q, w, nonstrict, variant)


def _instances(problems, op: str):
    """ctypes descriptors for (D, Q, w) CUDA tensors, the outputs, and the
    tensors the descriptors point into (to keep alive)."""
    torch = _torch()
    k = len(problems)
    arr = (domagg_instance * k)()
    outs, keep = [], []
    for i, (D, Q, w) in enumerate(problems):
        D, Q = D.contiguous(), Q.contiguous()
        w = None if op == "count" else w.contiguous()
        out = torch.empty(Q.shape[0], dtype=out_dtype(op, w), device=D.device)
        keep += [D, Q, w]
        outs.append(out)
        arr[i] = domagg_instance(D.shape[1], D.shape[0], Q.shape[0], D.data_ptr() if D.numel() else None,
                                 Q.data_ptr() if Q.numel() else None,
                                 w.data_ptr() if (w is not None and w.numel()) else None,
                                 out.data_ptr() if out.numel() else None)
    return arr, outs, keep


def batch(problems, op: str = "sum"):
    """problems: list of (D, Q, w) CUDA tensors (w ignored for count); all
    instances share coordinate dtype, weight dtype and op.  Returns outputs."""
    if not problems:
        return []
    arr, outs, keep = _instances(problems, op)
    D0 = problems[0][0]
    w0 = problems[0][2]
    dev = D0.device.index or 0
    domagg_batch(handle(dev), len(problems), arr, _coord_dtype(D0), _weight_dtype(w0, op), OPS[op],
                 _stream(D0.device))
    return outs


class BatchPlan:
    """A planned batch (domagg_batch_plan): `run()` enqueues one run of the
    batch on the current stream with no synchronisation, allocation or copy,
    so it can be captured in a CUDA graph.  The problems' tensors are kept
    alive by the plan; change their contents in place between runs.  `outs`
    holds the outputs (written by every run)."""

    def __init__(self, problems, op: str = "sum", headroom: float = 0.25):
        if not problems:
            raise ValueError("empty batch")
        self.arr, self.outs, self._keep = _instances(problems, op)
        D0 = problems[0][0]
        self.device = D0.device
        self._p = domagg_batch_plan(D0.device.index or 0, len(problems), self.arr, _coord_dtype(D0),
                                    _weight_dtype(problems[0][2], op), OPS[op], float(headroom),
                                    _stream(D0.device))

    def run(self):
        domagg_plan_run(self._p, _stream(self.device))

    def status(self):
        """Synchronises and raises DomaggError for a device-side error of the
        runs so far (e.g. more records than reserved)."""
        domagg_plan_status(self._p, _stream(self.device))

    def autotune(self) -> float:
        """Chooses the fastest launch shapes by timing runs (synchronises);
        returns the chosen shapes' time in ms."""
        return domagg_plan_autotune(self._p, _stream(self.device))

    def workspace_bytes(self) -> int:
        return domagg_plan_workspace_bytes(self._p)

    def close(self):
        if getattr(self, "_p", None):
            domagg_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stats(device: int = 0) -> dict:
    return domagg_get_stats(handle(device))
