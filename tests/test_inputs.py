"""Seeded input generators: valid CSR (sorted simple rows, symmetric, one
component), determinism, and the native R-MAT generator's independence of the
thread count."""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

from pw_inputs import (barabasi_albert, eps_choice, eps_uniform, er_cycle, grid_deleted, poisson_arrivals,
                       query_seeds, rmat, rmat_native, uniform_pairs)


def _check_csr(g):
    rp, ci = np.asarray(g.row_ptr), np.asarray(g.col_idx)
    assert rp[0] == 0 and rp[-1] == ci.size and np.all(np.diff(rp) >= 1)
    assert ci.min() >= 0 and ci.max() < g.n
    rows = np.repeat(np.arange(g.n), np.diff(rp))
    assert not np.any(rows == ci)  # no self-loops
    for v in range(0, g.n, max(1, g.n // 200)):  # rows strictly increasing (so no duplicates)
        r = ci[rp[v]:rp[v + 1]]
        assert np.all(np.diff(r) > 0)
    a = csr_matrix((np.ones(ci.size, np.int8), ci, rp), shape=(g.n, g.n))
    assert (a != a.T).nnz == 0  # symmetric
    assert connected_components(a, directed=False)[0] == 1


@pytest.mark.parametrize("make", [lambda: er_cycle(200, 8 / 199, 0), lambda: barabasi_albert(2000, 5, 1),
                                  lambda: rmat(12, 16, (0.57, 0.19, 0.19, 0.05), 2), lambda: grid_deleted(60, 0.05, 3),
                                  lambda: rmat_native(12, 16, (0.57, 0.19, 0.19, 0.05), 4)])
def test_generators_give_valid_connected_csr(make):
    g = make()
    _check_csr(g)
    again = make()
    assert np.array_equal(g.row_ptr, again.row_ptr) and np.array_equal(g.col_idx, again.col_idx)


def test_rmat_native_independent_of_thread_count():
    one = rmat_native(13, 16, (0.57, 0.19, 0.19, 0.05), 7, threads=1)
    four = rmat_native(13, 16, (0.57, 0.19, 0.19, 0.05), 7, threads=4)
    assert one.n == four.n
    assert np.array_equal(one.row_ptr, four.row_ptr) and np.array_equal(one.col_idx, four.col_idx)
    deg = np.diff(one.row_ptr)
    assert deg.max() > 20 * deg.mean()  # heavy-tailed, as R-MAT with (.57, .19, .19, .05) should be


def test_grid_is_bipartite_and_ba_is_not():
    assert grid_deleted(40, 0.05, 3).is_bipartite()
    assert not barabasi_albert(500, 3, 1).is_bipartite()


def test_query_streams_seeded():
    s, t = uniform_pairs(1000, 500, 11)
    s2, t2 = uniform_pairs(1000, 500, 11)
    assert np.array_equal(s, s2) and np.array_equal(t, t2)
    assert np.all(s != t) and s.min() >= 0 and max(s.max(), t.max()) < 1000
    e = eps_uniform(1000, 0.05, 0.2, 3)
    assert e.min() >= 0.05 and e.max() <= 0.2
    c = eps_choice(300, [0.05, 0.1, 0.2], 4)
    assert set(np.unique(c).tolist()) <= {0.05, 0.1, 0.2}
    q = query_seeds(100, 5)
    assert np.unique(q).size == 100
    arr = poisson_arrivals(2000, 100.0, 6)
    assert np.all(np.diff(arr) >= 0) and abs(arr[-1] / 2000 - 0.01) < 0.002
