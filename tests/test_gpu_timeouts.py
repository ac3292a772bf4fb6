"""Device-side wait limits: a wait on something that never happens gives up
after about a second, records DOMAGG_ERR_TIMEOUT for the host, and leaves
the context usable (no fault, no hang)."""
import time

import numpy as np
import pytest

from gpu_helpers import assert_matches_oracle, gpu_forward, torch
from paper_2305_16751_gb300 import domagg, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1], ids=["lookback", "mbarrier"])
def test_wait_gives_up_and_reports_timeout(which):
    t = torch()
    h = domagg.handle(0)
    stream = domagg._stream(t.device("cuda", 0))
    t0 = time.perf_counter()
    st = domagg.lib().domagg_selftest_timeout(h, which, stream)
    elapsed = time.perf_counter() - t0
    assert st == 5, domagg.lib().domagg_last_error(h).decode()  # DOMAGG_ERR_TIMEOUT
    assert 0.05 < elapsed < 30.0
    # the error was consumed and the handle still computes correctly
    assert domagg.lib().domagg_sync_status(h, stream) == 0
    rng = np.random.default_rng(9)
    D, Q, w = workloads.random_small(rng, 2, 3000, 2000, 50, "i32", "i64")
    assert_matches_oracle(gpu_forward(D, Q, w, "sum"), D, Q, w, "sum")
