"""The exchange step of the sharded forward on CPU ranks (gloo, two
processes): each rank holds the float-float partial outputs of its shard;
after the all-gather of paper_2305_16751_gb300.shards every rank has every
rank's parts in rank order, and their float-float sum is the exact total
(checked in float64).  The GPU join itself is covered by the -m gpu tests."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_2305_16751_gb300 import shards
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(100 + rank)
        exact = rng.standard_normal(1000) * 10.0 ** rng.integers(-3, 4, 1000)
        hi = exact.astype(np.float32)
        lo = (exact - hi.astype(np.float64)).astype(np.float32)
        parts = shards.gather(torch.from_numpy(hi))
        los = shards.gather(torch.from_numpy(lo))
        # every rank's parts, in rank order
        ok = True
        total = np.zeros(1000)
        for r in range(world):
            e = np.random.default_rng(100 + r)
            ex = e.standard_normal(1000) * 10.0 ** e.integers(-3, 4, 1000)
            got = parts[r].numpy().astype(np.float64) + los[r].numpy().astype(np.float64)
            ok &= bool(np.allclose(got, ex, rtol=2.0**-44, atol=0))
            total += got
        q.put((rank, ok, float(np.abs(total).sum())))
    finally:
        dist.destroy_process_group()


def test_two_ranks_exchange_float_float_partials():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert sorted(r for r, _, _ in res) == [0, 1]
    assert all(ok for _, ok, _ in res)
    assert res[0][2] == pytest.approx(res[1][2])
