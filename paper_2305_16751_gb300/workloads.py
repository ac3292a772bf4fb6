"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers.  It holds none of the method's
arithmetic, and it is the one piece that both the CUDA path's tests / bench
and the CPU oracle's tests use.  The paper runs no experiments (its summary
names experiments as future work), so every input is synthetic; the five
workloads below are the ones the library is measured and checked on.

All draws use numpy's PCG64 ``default_rng(seed)`` with
``seed = 2305167510 + workload index`` unless a seed is given.  Floats in
[0, 1) are drawn on a 24-bit grid, ``(u32 >> 8) * 2**-24``, so ties are
explicit and every value is exact in float32.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2305167510


@dataclass
class Problem:
    """One instance: data points D [nD, m], queries Q [nQ, m], weights w [nD]."""

    m: int
    D: np.ndarray
    Q: np.ndarray
    w: np.ndarray | None
    op: str
    name: str = ""
    extra: dict = field(default_factory=dict)


def _rng(index: int, seed: int | None) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + index if seed is None else seed)


def grid24(rng: np.random.Generator, shape) -> np.ndarray:
    """Uniform floats in [0, 1) on the 2^-24 grid (exact in float32)."""
    u = rng.integers(0, 2**32, size=shape, dtype=np.uint64)
    return ((u >> np.uint64(8)).astype(np.float64) * 2.0**-24).astype(np.float32)


def uniform_i32_coords(n: int, m: int, lo: int, hi: int, seed: int | None = None,
                       index: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """Two point sets [n, m] of int32 uniform in [lo, hi)."""
    rng = _rng(index, seed)
    D = rng.integers(lo, hi, size=(n, m), dtype=np.int64).astype(np.int32)
    Q = rng.integers(lo, hi, size=(n, m), dtype=np.int64).astype(np.int32)
    return D, Q


def small_int(n: int = 4096, m: int = 2, seed: int | None = None, op: str = "sum") -> Problem:
    """m=2, |D|=|Q|=4096, int32 coordinates uniform in [0, 2^20), int64
    weights uniform in [-1000, 1000] (sum and count)."""
    rng = _rng(1, seed)
    D = rng.integers(0, 2**20, size=(n, m), dtype=np.int64).astype(np.int32)
    Q = rng.integers(0, 2**20, size=(n, m), dtype=np.int64).astype(np.int32)
    w = rng.integers(-1000, 1001, size=n, dtype=np.int64)
    return Problem(m, D, Q, w, op, name=f"m{m}_n{n}_i32coords_i64w")


def tied_floats(n: int = 2**24, m: int = 2, seed: int | None = None, weights: str = "f32",
                quantised_fraction: float = 0.25) -> Problem:
    """m=2, |D|=|Q|=n, float32 coordinates uniform in [0, 1) on the 24-bit
    grid; a seeded Bernoulli(0.25) choice of points has all its coordinates
    rounded down to the 2^-16 grid, which forces ties within and between D and
    Q.  weights='f32': N(0, 1) float32 weights, F = sum; weights='i32': int32
    weights uniform in [-2^30, 2^30), F = max."""
    rng = _rng(2, seed)
    pts = []
    for _ in range(2):
        x = grid24(rng, (n, m))
        quant = rng.random(n) < quantised_fraction
        x[quant] = (np.floor(x[quant].astype(np.float64) * 2.0**16) * 2.0**-16).astype(np.float32)
        pts.append(x)
    if weights == "f32":
        w = rng.standard_normal(n, dtype=np.float32)
        op = "sum"
    elif weights == "i32":
        w = rng.integers(-2**30, 2**30, size=n, dtype=np.int64).astype(np.int32)
        op = "max"
    else:
        raise ValueError(weights)
    return Problem(m, pts[0], pts[1], w, op, name=f"m{m}_n{n}_f32tied_{weights}w_{op}")


def gaussian_mixture_i32(n: int = 2**21, m: int = 3, seed: int | None = None,
                         components: int = 16) -> Problem:
    """m=3, |D|=|Q|=n, int32 coordinates from a 16-component Gaussian mixture
    (means uniform in [0, 2^24), per-dimension sigma uniform in
    [2^16, 2^20]), rounded and clipped to [0, 2^24); int64 weights uniform in
    [0, 2^20), F = sum."""
    rng = _rng(3, seed)
    means = rng.uniform(0, 2**24, size=(components, m))
    sig = rng.uniform(2**16, 2**20, size=(components, m))
    pts = []
    for _ in range(2):
        comp = rng.integers(0, components, size=n)
        x = rng.standard_normal((n, m)) * sig[comp] + means[comp]
        x = np.clip(np.rint(x), 0, 2**24 - 1).astype(np.int32)
        pts.append(x)
    w = rng.integers(0, 2**20, size=n, dtype=np.int64)
    return Problem(m, pts[0], pts[1], w, "sum", name=f"m{m}_n{n}_gmm_i32coords_i64w")


def autograd_floats(n: int = 2**22, m: int = 2, seed: int | None = None) -> Problem:
    """m=2, |D|=|Q|=n, float32 coordinates uniform in [0, 1) (24-bit grid),
    float32 weights N(0, 1) and loss coefficients c ~ N(0, 1) for
    L = sum_q c_q out_q."""
    rng = _rng(4, seed)
    D = grid24(rng, (n, m))
    Q = grid24(rng, (n, m))
    w = rng.standard_normal(n, dtype=np.float32)
    c = rng.standard_normal(n, dtype=np.float32)
    return Problem(m, D, Q, w, "sum", name=f"m{m}_n{n}_f32_autograd", extra={"c": c})


def batch_sizes(k: int = 4096, lo: int = 256, hi: int = 2**18, seed: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Per-instance m (2 or 3, 50/50) and |D| = |Q| log-uniform in [lo, hi]."""
    rng = _rng(5, seed)
    ms = rng.integers(2, 4, size=k)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=k)).astype(np.int64)
    return ms, np.clip(sizes, lo, hi)


def batch_instances(k: int = 4096, lo: int = 256, hi: int = 2**18, seed: int | None = None) -> list[Problem]:
    """4096 independent instances, m in {2, 3} 50/50, |D| = |Q| log-uniform in
    [256, 2^18], int32 coordinates uniform in [0, 2^31), float32 weights
    N(0, 1), F = sum."""
    ms, sizes = batch_sizes(k, lo, hi, seed)
    rng = _rng(5, None if seed is None else seed + 1)
    out = []
    for i in range(k):
        n, m = int(sizes[i]), int(ms[i])
        D = rng.integers(0, 2**31, size=(n, m), dtype=np.int64).astype(np.int32)
        Q = rng.integers(0, 2**31, size=(n, m), dtype=np.int64).astype(np.int32)
        w = rng.standard_normal(n, dtype=np.float32)
        out.append(Problem(m, D, Q, w, "sum", name=f"batch{i}"))
    return out


def ecdf_samples(n: int = 2**20, m: int = 3, shift: float = 0.05, seed: int | None = None) -> Problem:
    """Two samples for the empirical CDF / two-sample statistic (dominance
    counting with every coordinate non-strict): X ~ N(0, 1)^m in D, Y ~
    N(shift, 1)^m in Q, float32 on a 2^-8 grid (ties within and across the
    samples)."""
    rng = _rng(6, seed)
    X = (np.round(rng.standard_normal((n, m)) * 256.0) / 256.0).astype(np.float32)
    Y = (np.round((rng.standard_normal((n, m)) + shift) * 256.0) / 256.0).astype(np.float32)
    return Problem(m=m, D=X, Q=Y, w=None, op="count", name=f"ecdf_m{m}_n{n}")


def random_small(rng: np.random.Generator, m: int, nD: int, nQ: int, levels: int, dtype: str,
                 weights: str) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Tiny random cases with heavy ties: every coordinate is an integer in
    [-ceil(levels/2), ceil(levels/2)) -- `levels` values for even `levels`,
    one more for odd -- as int32, or halved as float32 (negative values
    included)."""
    vals = rng.integers(-levels // 2, levels - levels // 2, size=(nD + nQ, m))
    if dtype == "f32":
        pts = (vals.astype(np.float32) * np.float32(0.5))
    else:
        pts = vals.astype(np.int32)
    D, Q = pts[:nD].copy(), pts[nD:].copy()
    if weights == "i64":
        w = rng.integers(-1000, 1001, size=nD, dtype=np.int64)
    elif weights == "i32":
        w = rng.integers(-2**30, 2**30, size=nD, dtype=np.int64).astype(np.int32)
    else:
        w = rng.standard_normal(nD).astype(np.float32)
    return D, Q, w
