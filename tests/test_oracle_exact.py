"""Pins for the exact oracle (Definition 2.1) and the truncated series (Lemma 2.3).

Closed forms come from the Laplacian spectra of complete, cycle and path graphs;
invariants come from Eq. exact (beta is a squared Euclidean norm), the range
n^-2 <= beta <= n^3 quoted in Section 2.2, Lemma 3.5 and its R_eff step.
"""

import math

import numpy as np
import pytest

from oracle import exact
from pw_inputs import barabasi_albert, complete_graph, cycle_graph, er_cycle, grid_deleted, path_graph


def cycle_closed_form(n, delta):
    # L of C_n has eigenvalues 2 - 2cos(2 pi k / n) with Fourier eigenvectors
    return sum((2 - 2 * math.cos(2 * math.pi * k * delta / n)) / n / (2 - 2 * math.cos(2 * math.pi * k / n)) ** 2
               for k in range(1, n))


def path_closed_form(n, s, t):
    # L of P_n has eigenvalues 2 - 2cos(pi k / n), eigenvectors sqrt(2/n) cos(pi k (j + 1/2) / n)
    tot = 0.0
    for k in range(1, n):
        mu = 2 - 2 * math.cos(math.pi * k / n)
        us = math.sqrt(2 / n) * math.cos(math.pi * k * (s + 0.5) / n)
        ut = math.sqrt(2 / n) * math.cos(math.pi * k * (t + 0.5) / n)
        tot += (us - ut) ** 2 / mu**2
    return tot


@pytest.mark.parametrize("n", [3, 4, 7, 10, 12])
def test_complete_graph(n):
    g = complete_graph(n)
    m = exact.exact_beta_matrix(g.row_ptr, g.col_idx, n)
    off = m[~np.eye(n, dtype=bool)]
    np.testing.assert_allclose(off, 2.0 / n**2, rtol=1e-11)


@pytest.mark.parametrize("n", [5, 8, 9, 12])
def test_cycle_graph(n):
    g = cycle_graph(n)
    for delta in range(1, n):
        got = exact.exact_beta(g.row_ptr, g.col_idx, n, 0, delta)
        assert got == pytest.approx(cycle_closed_form(n, delta), rel=1e-10)


def test_cycle9_rationals():
    # The C_9 closed form sums to 20/27, 56/27 and 110/27 at distances 1, 2 and 4.
    g = cycle_graph(9)
    for delta, frac in ((1, 20 / 27), (2, 56 / 27), (4, 110 / 27)):
        assert exact.exact_beta(g.row_ptr, g.col_idx, 9, 0, delta) == pytest.approx(frac, rel=1e-12)


@pytest.mark.parametrize("n", [2, 3, 6, 10])
def test_path_graph(n):
    g = path_graph(n)
    for s in range(n):
        for t in range(n):
            got = exact.exact_beta(g.row_ptr, g.col_idx, n, s, t)
            assert got == pytest.approx(path_closed_form(n, s, t), rel=1e-10, abs=1e-12)
    # end to end of P_6 is 35/2
    if n == 6:
        assert exact.exact_beta(g.row_ptr, g.col_idx, 6, 0, 5) == pytest.approx(17.5, rel=1e-12)


def _small_graphs():
    yield er_cycle(200, 8 / 199, 0)
    yield er_cycle(60, 0.1, 5)
    yield barabasi_albert(120, 2, 9)
    yield grid_deleted(8, 0.1, 4)


@pytest.mark.parametrize("g", list(_small_graphs()), ids=lambda g: g.name)
def test_invariants(g):
    n = g.n
    m = exact.exact_beta_matrix(g.row_ptr, g.col_idx, n)
    assert np.allclose(np.diag(m), 0.0, atol=1e-12)            # beta(s,s) = 0
    assert np.allclose(m, m.T, rtol=1e-12, atol=1e-14)          # symmetry
    off = m[~np.eye(n, dtype=bool)]
    assert off.min() >= n**-2.0 * (1 - 1e-9) and off.max() <= n**3.0  # range of Section 2.2
    b = np.sqrt(np.maximum(m, 0))
    rng = np.random.default_rng(0)
    tri = rng.integers(0, n, size=(2000, 3))
    x, y, z = tri.T
    assert np.all(b[x, z] <= b[x, y] + b[y, z] + 1e-9)           # b is a Euclidean distance
    deg = g.degrees.astype(float)
    lp = exact.laplacian_pinv(g.row_ptr, g.col_idx, n)
    reff = np.diag(lp)[:, None] + np.diag(lp)[None, :] - 2 * lp
    lower = 0.125 * (1 / deg[:, None] + 1 / deg[None, :]) ** 2
    mask = ~np.eye(n, dtype=bool)
    assert np.all(m[mask] >= reff[mask] ** 2 / 2 * (1 - 1e-9))   # Cauchy-Schwarz step of Lemma 3.5
    assert np.all(m[mask] >= lower[mask] * (1 - 1e-9))           # Lemma 3.5


def test_pinv_identity(tiny_graph):
    g = tiny_graph
    lp = exact.laplacian_pinv(g.row_ptr, g.col_idx, g.n)
    a = np.zeros((g.n, g.n))
    a[np.repeat(np.arange(g.n), g.degrees), g.col_idx] = 1
    lap = np.diag(a.sum(1)) - a
    # Moore-Penrose conditions
    assert np.allclose(lap @ lp @ lap, lap, atol=1e-10)
    assert np.allclose(lp @ lap @ lp, lp, atol=1e-10)
    assert np.allclose(lp.sum(axis=0), 0.0, atol=1e-10)


# ---------------------------------------------------------------- series


@pytest.mark.parametrize("n", [3, 5, 10])
@pytest.mark.parametrize("L", [0, 1, 2, 5, 17])
def test_series_complete_graph(n, L):
    # P^i D^-1 b = (-1/(n-1))^i b / (n-1) on K_n, so beta^(L) = (2/n^2)(1 - (-1/(n-1))^(L+1))^2
    g = complete_graph(n)
    want = 2.0 / n**2 * (1 - (-1.0 / (n - 1)) ** (L + 1)) ** 2
    assert exact.series_beta(g.row_ptr, g.col_idx, n, 0, n - 1, L) == pytest.approx(want, rel=1e-12)


def test_series_L0(tiny_graph):
    g = tiny_graph
    d = g.degrees.astype(float)
    for s, t in ((0, 1), (3, 77), (150, 9)):
        want = 1 / d[s] ** 2 + 1 / d[t] ** 2 - (1 / d[s] - 1 / d[t]) ** 2 / g.n
        assert exact.series_beta(g.row_ptr, g.col_idx, g.n, s, t, 0) == pytest.approx(want, rel=1e-13)


def test_series_many_matches_single(tiny_graph):
    g = tiny_graph
    s = np.array([0, 3, 150])
    t = np.array([1, 77, 9])
    many = exact.series_beta_many(g.row_ptr, g.col_idx, g.n, s, t, 12)
    for i in range(3):
        assert many[i] == pytest.approx(exact.series_beta(g.row_ptr, g.col_idx, g.n, s[i], t[i], 12), rel=1e-12)


@pytest.mark.parametrize("g", [er_cycle(200, 8 / 199, 0), er_cycle(60, 0.1, 5), barabasi_albert(120, 2, 9)],
                         ids=lambda g: g.name)
def test_truncation_bound_lemma_2_3(g):
    """|beta - beta^(L)| <= eta/2 at the L of Eq. uni_l (non-bipartite graphs)."""
    assert not g.is_bipartite()
    lam = exact.mixing_lambda(g.row_ptr, g.col_idx, g.n)
    m = exact.exact_beta_matrix(g.row_ptr, g.col_idx, g.n)
    rng = np.random.default_rng(1)
    for eta in (1e-2, 1e-4):
        L = exact.truncation_length(g.n, lam, eta)
        for _ in range(5):
            s, t = rng.choice(g.n, 2, replace=False)
            bl = exact.series_beta(g.row_ptr, g.col_idx, g.n, int(s), int(t), L)
            assert abs(m[s, t] - bl) <= eta / 2


def test_series_converges_to_exact(tiny_graph):
    g = tiny_graph
    ex = exact.exact_beta(g.row_ptr, g.col_idx, g.n, 3, 77)
    errs = [abs(exact.series_beta(g.row_ptr, g.col_idx, g.n, 3, 77, L) - ex) for L in (4, 8, 16, 32, 64)]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-12 * max(1.0, ex) + 1e-14


def test_bipartite_grid_series_oscillates():
    """On a bipartite graph P has eigenvalue -1, so for s, t of opposite colour
    beta^(L) keeps alternating instead of converging (Section 2.1 assumes a
    non-bipartite graph)."""
    g = path_graph(6)
    assert g.is_bipartite()
    even = exact.series_beta(g.row_ptr, g.col_idx, 6, 0, 1, 400)
    odd = exact.series_beta(g.row_ptr, g.col_idx, 6, 0, 1, 401)
    assert abs(even - odd) > 1e-3


# ---------------------------------------------------------------------------
# Effective resistance (proof of Lemma 3.5) and the mixing parameter lambda
# (Section 2.1), pinned by closed forms and Foster's theorem.  The helpers take
# the module so that planted mistakes in a copy of it can be run through them.
# ---------------------------------------------------------------------------

def circulant(n, steps):
    u = np.concatenate([np.arange(n)] * len(steps))
    v = np.concatenate([(np.arange(n) + s) % n for s in steps])
    from pw_inputs import from_edges

    return from_edges(n, u, v, name=f"circ{n}")


def petersen():
    from pw_inputs import from_edges

    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    e = np.array(outer + spokes + inner)
    return from_edges(10, e[:, 0], e[:, 1], name="petersen")


def check_effective_resistance(ex):
    for n in (3, 5, 8):  # K_n: 2/n
        g = complete_graph(n)
        assert ex.effective_resistance(g.row_ptr, g.col_idx, n, 0, n - 1) == pytest.approx(2 / n, rel=1e-11)
    for n in (2, 5, 9):  # P_n: resistors in series, |s - t|
        g = path_graph(n)
        for s, t in ((0, n - 1), (1, n // 2)):
            assert ex.effective_resistance(g.row_ptr, g.col_idx, n, s, t) == pytest.approx(abs(s - t), rel=1e-10,
                                                                                          abs=1e-12)
    for n in (4, 7, 10):  # C_n: paths of k and n - k edges in parallel, k (n - k) / n
        g = cycle_graph(n)
        for k in range(1, n):
            assert ex.effective_resistance(g.row_ptr, g.col_idx, n, 0, k) == pytest.approx(k * (n - k) / n, rel=1e-10)
    # Foster's theorem: the effective resistances of the edges sum to n - 1
    for g in (er_cycle(30, 0.2, 4), barabasi_albert(40, 2, 9), petersen()):
        src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        tot = sum(ex.effective_resistance(g.row_ptr, g.col_idx, g.n, int(a), int(b))
                  for a, b in zip(src, g.col_idx) if a < b)
        assert tot == pytest.approx(g.n - 1, rel=1e-10)


def check_mixing_lambda(ex):
    for n in (3, 5, 10):  # K_n: P = (J - I)/(n - 1), eigenvalues 1 and -1/(n - 1)
        g = complete_graph(n)
        assert ex.mixing_lambda(g.row_ptr, g.col_idx, n) == pytest.approx(1 / (n - 1), rel=1e-11)
    for n in (5, 7, 9, 15):  # odd C_n: eigenvalues cos(2 pi k / n); the largest |.| for k >= 1 is cos(pi / n)
        g = cycle_graph(n)
        assert ex.mixing_lambda(g.row_ptr, g.col_idx, n) == pytest.approx(math.cos(math.pi / n), rel=1e-11)
    for n in (4, 6, 10):  # even C_n is bipartite: -1 is an eigenvalue
        g = cycle_graph(n)
        assert ex.mixing_lambda(g.row_ptr, g.col_idx, n) == pytest.approx(1.0, rel=1e-11)
    g = petersen()  # adjacency spectrum {3, 1, -2}: P has 1, 1/3, -2/3
    assert ex.mixing_lambda(g.row_ptr, g.col_idx, 10) == pytest.approx(2 / 3, rel=1e-11)
    for n in (12, 20):  # circulant C_n(1, 2): eigenvalues (cos(2 pi k/n) + cos(4 pi k/n)) / 2
        g = circulant(n, (1, 2))
        want = max(abs(math.cos(2 * math.pi * k / n) + math.cos(4 * math.pi * k / n)) / 2 for k in range(1, n))
        assert ex.mixing_lambda(g.row_ptr, g.col_idx, n) == pytest.approx(want, rel=1e-11)


def test_effective_resistance_closed_forms():
    check_effective_resistance(exact)


def test_mixing_lambda_closed_forms():
    check_mixing_lambda(exact)


# ---------------------------------------------------------------------------
# The same closed forms for beta, L^+ and the series, taking the module, so
# that planted mistakes in a copy of it can be run through them.
# ---------------------------------------------------------------------------


def check_exact_beta(ex):
    for n in (4, 7):  # K_n: 2/n^2 off the diagonal, 0 on it
        g = complete_graph(n)
        m = ex.exact_beta_matrix(g.row_ptr, g.col_idx, n)
        np.testing.assert_allclose(m[~np.eye(n, dtype=bool)], 2.0 / n**2, rtol=1e-11)
        np.testing.assert_allclose(np.diag(m), 0.0, atol=1e-12)
    g = cycle_graph(9)  # C_9 closed form: 20/27, 56/27, 110/27
    for delta, frac in ((1, 20 / 27), (2, 56 / 27), (4, 110 / 27)):
        assert ex.exact_beta(g.row_ptr, g.col_idx, 9, 0, delta) == pytest.approx(frac, rel=1e-12)
    g = path_graph(6)  # end to end of P_6: 35/2
    assert ex.exact_beta(g.row_ptr, g.col_idx, 6, 0, 5) == pytest.approx(17.5, rel=1e-12)
    g = er_cycle(40, 0.15, 2)  # Moore-Penrose conditions of L^+
    lp = ex.laplacian_pinv(g.row_ptr, g.col_idx, g.n)
    a = np.zeros((g.n, g.n))
    a[np.repeat(np.arange(g.n), g.degrees), g.col_idx] = 1
    lap = np.diag(a.sum(1)) - a
    assert np.allclose(lap @ lp @ lap, lap, atol=1e-10)
    assert np.allclose(lp @ lap @ lp, lp, atol=1e-10)
    assert np.allclose(lp, lp.T, atol=1e-12)


def check_series(ex):
    for n, L in ((3, 0), (5, 1), (10, 5)):  # K_n: (2/n^2)(1 - (-1/(n-1))^(L+1))^2
        g = complete_graph(n)
        want = 2.0 / n**2 * (1 - (-1.0 / (n - 1)) ** (L + 1)) ** 2
        assert ex.series_beta(g.row_ptr, g.col_idx, n, 0, n - 1, L) == pytest.approx(want, rel=1e-12)
    g = er_cycle(40, 0.15, 2)  # L = 0 closed form on an irregular graph
    d = g.degrees.astype(float)
    for s, t in ((0, 1), (3, 27)):
        want = 1 / d[s] ** 2 + 1 / d[t] ** 2 - (1 / d[s] - 1 / d[t]) ** 2 / g.n
        assert ex.series_beta(g.row_ptr, g.col_idx, g.n, s, t, 0) == pytest.approx(want, rel=1e-13)
    ref = exact.exact_beta(g.row_ptr, g.col_idx, g.n, 3, 27)  # converges to beta (non-bipartite)
    assert ex.series_beta(g.row_ptr, g.col_idx, g.n, 3, 27, 400) == pytest.approx(ref, rel=1e-9)
    # the many-pair form: the same closed forms, column by column
    many = ex.series_beta_many(g.row_ptr, g.col_idx, g.n, np.array([0, 3]), np.array([1, 27]), 0)
    for i, (s, t) in enumerate(((0, 1), (3, 27))):
        want = 1 / d[s] ** 2 + 1 / d[t] ** 2 - (1 / d[s] - 1 / d[t]) ** 2 / g.n
        assert many[i] == pytest.approx(want, rel=1e-13)
    k = complete_graph(6)
    many = ex.series_beta_many(k.row_ptr, k.col_idx, 6, np.array([0, 2]), np.array([5, 3]), 3)
    np.testing.assert_allclose(many, 2.0 / 36 * (1 - (-1.0 / 5) ** 4) ** 2, rtol=1e-12)


def test_exact_beta_checks():
    check_exact_beta(exact)


def test_series_checks():
    assert not er_cycle(40, 0.15, 2).is_bipartite()
    check_series(exact)
