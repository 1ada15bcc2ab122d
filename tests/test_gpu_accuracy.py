"""Problem 1's accuracy target on the larger workloads: at least 95% of the
queries within eps of the truncated distance beta^(L) (Theorem 3.8 gives it
with probability 1 - delta per query), with the default PILOT budget.  The
reference beta^(L) comes from pw_series_batch, which test_gpu_parity pins to
the oracle's FP64 series at 1e-9.  The query sets are the workloads' own seeded
pairs, so each fraction is deterministic."""

import numpy as np
import pytest

from pw_inputs import query_seeds, rmat, uniform_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_2512_05460_gb300 import build

    build.build()
    from paper_2512_05460_gb300 import probewalk

    probewalk.lib()
    return probewalk


def test_rmat20_accuracy_1024_queries(pw):
    """R-MAT 2^20 (646K nodes, hubs of degree ~10^4), L = 500, eps = 0.2:
    1024 uniform pairs; about 11% of them have their R clamped at R_max."""
    host = rmat(20, 16, (0.57, 0.19, 0.19, 0.05), 2)
    n = 1024
    s, t = uniform_pairs(host.n, n, 102)
    seeds = query_seeds(n, 1002)
    with pw.Graph(host.row_ptr, host.col_idx) as g:
        ref = pw.pw_series_batch(g.handle, s, t, np.full(n, 500, np.int32))
        beta, st = pw.pw_query_batch(g.handle, s, t, 0.2, 500, seeds)
    assert np.all(st == 0) and np.all(ref > 0)
    within = np.abs(beta - ref) / ref <= 0.2
    assert within.mean() >= 0.95, within.mean()
