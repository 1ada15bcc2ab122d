"""Pins for the oracle's Paired-Sign Probe generator (Definition 3.1, Section 3.3).

Structure: pi_k is a permutation of [n]; |U| = r with r = 1 for odd n and
r in {0, 2} by a fair coin for even n; paired entries have opposite signs, so
sum(z) = 0; the partner map is a fixed-point-free involution on the active set.
Statistics: E[z z^T] = H (Lemma 3.2) within CLT bounds.  Brute force: the
ideal probe distribution gives E[phi(z)^2] = beta^(L) exactly (Lemma 3.3),
and the generator's probes reproduce it within CLT bounds.
"""

import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import exact
from pw_inputs import barabasi_albert, complete_graph, er_cycle, from_edges, path_graph


@pytest.mark.parametrize("n", [2, 3, 4, 5, 16, 17, 63, 64, 65, 200, 1000, 4097])
def test_pi_is_permutation(oracle_lib, n):
    for seed, k in ((1, 0), (99, 7), (2**63 + 5, 123456)):
        z, pi, r = oracle.probe_vector(n, seed, k)
        assert sorted(pi.tolist()) == list(range(n))


@pytest.mark.parametrize("n", [2, 3, 7, 8, 10, 199, 200, 1001])
def test_probe_structure(oracle_lib, n):
    rs = set()
    for k in range(60):
        z, pi, r = oracle.probe_vector(n, 31337, k)
        rs.add(r)
        assert r == 1 if n % 2 else r in (0, 2)
        assert int((z == 0).sum()) == r
        assert np.all((z == 0) == (pi >= n - r))
        assert int(z.astype(np.int64).sum()) == 0
        inv = np.empty(n, np.int64)
        inv[pi.astype(np.int64)] = np.arange(n)
        active = np.flatnonzero(z != 0)
        partner = inv[pi[active].astype(np.int64) ^ 1]
        assert np.all(partner != active)                    # no fixed points
        assert np.all(inv[pi[partner].astype(np.int64) ^ 1] == active)  # involution
        assert np.all(z[partner] == -z[active])             # opposite signs within a pair
    if n % 2 == 0:
        assert rs == {0, 2}


def test_parity_coin_is_fair(oracle_lib):
    rs = np.array([oracle.probe_vector(10, 4242, k)[2] for k in range(4000)])
    frac = (rs == 2).mean()
    assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / 4000)


def _probes(n, m, seed):
    z = np.empty((m, n), np.int8)
    pi = np.empty((m, n), np.int64)
    r = np.empty(m, np.int64)
    for k in range(m):
        zk, pk, rk = oracle.probe_vector(n, seed, k)
        z[k], pi[k], r[k] = zk, pk.astype(np.int64), rk
    return z, pi, r


@pytest.mark.parametrize("n", [5, 7, 8, 10, 17, 20, 33, 100])
def test_second_moment_lemma_3_2(oracle_lib, n):
    """E[z z^T] = I - 11^T/n within 5 standard errors per entry (|z_i z_j| <= 1)."""
    m = 60000
    z, _, _ = _probes(n, m, 777)
    zf = z.astype(np.float64)
    emp = zf.T @ zf / m
    h = np.eye(n) - 1.0 / n
    assert np.max(np.abs(emp - h)) < 5 / math.sqrt(m)


@pytest.mark.parametrize("n", [5, 6, 7, 8, 10, 17, 20, 33, 100])
def test_pairing_is_uniform(oracle_lib, n):
    """The matching behind z is uniform: P(i, j paired) = (n - r)/(n (n - 1)) for every
    pair, averaged over r (the identity inside the proof of Lemma 3.2)."""
    m = 60000
    _, pi, r = _probes(n, m, 99)
    inv = np.argsort(pi, axis=1)
    act = pi < (n - r)[:, None]
    partner = np.take_along_axis(inv, np.minimum(pi ^ 1, n - 1), axis=1)
    rows = np.broadcast_to(np.arange(n), (m, n))
    counts = np.bincount(rows[act] * n + partner[act], minlength=n * n).reshape(n, n) / m
    want = (1 - 1 / n) / (n - 1)
    off = counts[~np.eye(n, dtype=bool)]
    se = math.sqrt(want / m)
    assert np.max(np.abs(off - want)) < 5.5 * se
    # marginals: P(i in U) = E[r]/n
    assert np.max(np.abs((~act).mean(0) - 1 / n)) < 5.5 * math.sqrt(1 / n / m)


def _perfect_matchings(items):
    if not items:
        yield []
        return
    first = items[0]
    for i in range(1, len(items)):
        rest = items[1:i] + items[i + 1:]
        for m in _perfect_matchings(rest):
            yield [(first, items[i])] + m


def ideal_probe_second_moment(h):
    """E[(z^T h)^2] under Definition 3.1, enumerated exactly."""
    n = len(h)
    total = 0.0
    r_choices = [(1, 1.0)] if n % 2 else [(0, 0.5), (2, 0.5)]
    for r, pr in r_choices:
        subsets = list(itertools.combinations(range(n), r))
        for U in subsets:
            rest = [i for i in range(n) if i not in U]
            matchings = list(_perfect_matchings(rest))
            for M in matchings:
                # signs independent per pair: E[(sum_e s_e (h_i - h_j))^2] = sum_e (h_i - h_j)^2
                val = sum((h[i] - h[j]) ** 2 for i, j in M)
                total += pr / len(subsets) / len(matchings) * val
    return total


@pytest.mark.parametrize("g", [complete_graph(5), path_graph(6), er_cycle(7, 0.4, 3),
                               from_edges(8, [0, 1, 2, 3, 4, 5, 6, 7, 0, 2], [1, 2, 3, 4, 5, 6, 7, 0, 4, 6], keep_lcc=False)],
                         ids=lambda g: g.name or f"n{g.n}")
@pytest.mark.parametrize("L", [0, 2, 5])
def test_lemma_3_3_brute_force(g, L):
    """beta^(L) = E_z[(z^T h^(L))^2] over the ideal Paired-Sign Probe."""
    s, t = 0, g.n - 2
    h = exact.series_h(g.row_ptr, g.col_idx, g.n, s, t, L)
    want = exact.series_beta(g.row_ptr, g.col_idx, g.n, s, t, L)
    assert ideal_probe_second_moment(h) == pytest.approx(want, rel=1e-11, abs=1e-15)


def test_generator_reproduces_lemma_3_3(oracle_lib):
    """The stateless generator's probes give E[phi(z)^2] = beta^(L) within CLT bounds."""
    g = barabasi_albert(50, 2, 3)
    s, t, L = 0, 31, 6
    h = exact.series_h(g.row_ptr, g.col_idx, g.n, s, t, L)
    want = exact.series_beta(g.row_ptr, g.col_idx, g.n, s, t, L)
    m = 40000
    vals = np.array([float(oracle.probe_vector(g.n, 5150, k)[0].astype(np.float64) @ h) ** 2 for k in range(m)])
    se = vals.std() / math.sqrt(m)
    assert abs(vals.mean() - want) < 5 * se
