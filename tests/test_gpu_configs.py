"""Parity at the larger workload sizes, in the launch configuration the
library picks for them: R-MAT 2^20 (646K nodes, 31M entries; split layout,
walk kernel per query), the 2000x2000 grid with 5% of edges deleted (4M
nodes; split layout; table too large for shared memory, per-visit kernel) and
R-MAT 2^24 (fused records: its split arrays would not fit L2 either).
The oracle recomputes sampled probes one by one."""

import numpy as np
import pytest

import oracle
from pw_inputs import eps_choice, eps_uniform, grid_deleted, query_seeds, rmat, uniform_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_2512_05460_gb300 import build

    build.build()
    from paper_2512_05460_gb300 import probewalk

    probewalk.lib()
    return probewalk


def _sampled_parity(pw, host, s, t, eps, L, seeds, n_sel=6, layout=None):
    with pw.Graph(host.row_ptr, host.col_idx) as g:
        if layout is not None:
            assert pw.pw_profile(g.handle, enable=False)["layout"] == layout
        rng = np.random.default_rng(5)
        sel_q = rng.integers(0, s.size, size=n_sel)
        sel_k = np.zeros(n_sel, np.int64)  # probe 0 exists for every query; resampled below
        beta, st, KR, _ = pw.pw_debug_batch_probe_q(g.handle, s, t, eps, L, seeds, sel_q, sel_k)
        assert np.all(st == 0) and np.all(np.isfinite(beta))
        sel_k = np.array([rng.integers(0, int(KR[q, 0])) for q in sel_q])
        beta2, _, KR2, qsel = pw.pw_debug_batch_probe_q(g.handle, s, t, eps, L, seeds, sel_q, sel_k)
        np.testing.assert_array_equal(beta2, beta)  # same batch twice: deterministic
        for i, (qi, k) in enumerate(zip(sel_q, sel_k)):
            b = oracle.budget(host, int(s[qi]), int(t[qi]), float(eps[qi]), int(L[qi]), int(seeds[qi]))
            assert (b["K"], b["R"]) == (int(KR[qi, 0]), int(KR[qi, 1]))
            want = oracle.probe_q(host, int(s[qi]), int(t[qi]), int(L[qi]), int(seeds[qi]), b["R"], [k])[0]
            assert qsel[i] == want


def test_rmat20_sampled_probes(pw, oracle_lib):
    host = rmat(20, 16, (0.57, 0.19, 0.19, 0.05), 2)
    s, t = uniform_pairs(host.n, 4, 102)
    eps = eps_uniform(4, 0.05, 0.2, 102)
    _sampled_parity(pw, host, s, t, eps, np.full(4, 500, np.int32), query_seeds(4, 1002), layout=2)


def test_grid_sampled_probes(pw, oracle_lib):
    host = grid_deleted(2000, 0.05, 3)
    assert host.is_bipartite()
    s, t = uniform_pairs(host.n, 4, 103)
    eps = eps_choice(4, [0.05, 0.1, 0.2], 103)
    _sampled_parity(pw, host, s, t, eps, np.full(4, 2000, np.int32), query_seeds(4, 1003), layout=2)


def test_rmat24_sampled_probes(pw, oracle_lib):
    """The scale configuration: R-MAT 2^24 (native generator, ~2.7e8 CSR entries,
    4.3 GB of records), L = 1000, eps uniform in [0.05, 0.2]."""
    from pw_inputs import rmat_native

    host = rmat_native(24, 16, (0.57, 0.19, 0.19, 0.05), 4)
    s, t = uniform_pairs(host.n, 3, 104)
    eps = eps_uniform(3, 0.05, 0.2, 104)
    _sampled_parity(pw, host, s, t, eps, np.full(3, 1000, np.int32), query_seeds(3, 1004), n_sel=4, layout=1)
