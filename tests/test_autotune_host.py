"""Host logic of the autotuner, on the CPU: every candidate is a tuning the
library accepts (tc_set_tuning checks the ranges without a device), and the
workload key is coarse (graphs, log2 of the median edges and of the mean
degree) and independent of the order of the graphs."""
import numpy as np
import pytest

import paper_1503_00576_gb300 as tc
from paper_1503_00576_gb300 import autotune

pytestmark = pytest.mark.usefixtures("libtc")


def test_candidates_are_valid_tunings():
    try:
        for c in autotune.CANDIDATES:
            tc.tc_set_tuning(c)
            assert tc.tc_get_tuning() == c
    finally:
        tc.tc_set_tuning(None)
    assert tc.tc_get_tuning() == tc.DEFAULT_TUNING
    assert autotune.CANDIDATES[0] == tc.DEFAULT_TUNING
    assert len({tuple(sorted(c.items())) for c in autotune.CANDIDATES}) == len(autotune.CANDIDATES)


def test_workload_key_is_coarse_and_order_free():
    rng = np.random.default_rng(3)
    m = rng.integers(1000, 3000, 64)
    n = rng.integers(100, 300, 64)
    eo = np.concatenate([[0], np.cumsum(m)])
    k = autotune.workload_key(eo, n)
    perm = rng.permutation(64)
    assert autotune.workload_key(np.concatenate([[0], np.cumsum(m[perm])]), n[perm]) == k
    assert k.startswith("g64/")
    # twice the edges on the same vertices: a different key
    eo2 = np.concatenate([[0], np.cumsum(4 * m)])
    assert autotune.workload_key(eo2, n) != k
