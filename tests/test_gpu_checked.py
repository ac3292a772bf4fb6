"""The checked build (DOMAGG_CHECKED): every kernel tests the indices it
loads and stores through and reports DOMAGG_ERR_BOUNDS instead of touching
memory outside a buffer.  The small parity cases run through it in a fresh
process, for every path (records pipeline, groups in shared memory, m = 3,
the level-wise formulation, the backward, a batch), with status OK and
results equal to the oracle's."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, torch, oracle
from paper_2305_16751_gb300 import domagg, workloads
assert "checked" in domagg.domagg_version(), domagg.domagg_version()
rng = np.random.default_rng(51)
dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
cases = []
for m in (1, 2, 3):
    for levels in (7, 3000, 1 << 20):
        D, Q, w = workloads.random_small(rng, m, 9001, 7003, levels, "f32", "i64")
        cases.append((D, Q, w))
for D, Q, w in cases:
    for op, ww in (("sum", w), ("count", None), ("max", w.astype(np.int32))):
        for variant in ("improved", "wavelet") if D.shape[1] <= 2 else ("improved",):
            got = domagg.forward(dev(D), dev(Q), dev(ww), op, variant=variant).cpu().numpy()
            want, _ = oracle.brute(D, Q, ww, op)
            assert np.array_equal(got.astype(np.int64), want.astype(np.int64)), (D.shape, op, variant)
    domagg.domagg_sync_status(domagg.handle(0), None)
p = workloads.tied_floats(n=1 << 18)
got = domagg.forward(dev(p.D), dev(p.Q), dev(p.w), "sum").cpu().numpy()
want, S = oracle.sweep2(p.D, p.Q, p.w, "sum")
assert np.all(np.abs(got - want) <= 4 * 2.0**-24 * S)
g = rng.standard_normal(p.Q.shape[0]).astype(np.float32)
gw = domagg.backward(dev(p.D), dev(p.Q), dev(g)).cpu().numpy()
wt, St = oracle.sweep2_transpose(p.D, p.Q, g)
assert np.all(np.abs(gw - wt) <= 4 * 2.0**-24 * St)
probs = [workloads.random_small(rng, 2, 3000, 2500, 500, "i32", "i64") for _ in range(6)]
outs = domagg.batch([(dev(D), dev(Q), dev(w)) for D, Q, w in probs], "sum")
for (D, Q, w), o in zip(probs, outs):
    assert np.array_equal(o.cpu().numpy(), oracle.brute(D, Q, w, "sum")[0])
domagg.domagg_sync_status(domagg.handle(0), None)
print("CHECKED OK")
"""


def test_checked_build_runs_the_parity_cases_clean():
    env = dict(os.environ, DOMAGG_CHECKED="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "CHECKED OK" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
