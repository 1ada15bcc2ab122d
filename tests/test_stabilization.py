"""The stabilization rule of Section 4.3 (oracle side, CPU): start at L = 1,
double L, accept L_stop = 2L once |beta(2L) - beta(L)| <= (eps/2)|beta(2L)|."""

import numpy as np
import pytest

import oracle
from oracle import exact
from pw_inputs import query_seeds, uniform_pairs


def test_rule_on_a_prescribed_sequence(monkeypatch, oracle_lib):
    seq = {1: 1.0, 2: 1.5, 4: 1.6, 8: 1.61, 16: 9.0}

    def fake_query(g, s, t, eps, L, seed, cfg=None, **kw):
        return {"beta": seq[L]}

    monkeypatch.setattr(oracle, "query", fake_query)
    # |1.6 - 1.5| = 0.1 > 0.05 * 1.6; |1.61 - 1.6| = 0.01 <= 0.05 * 1.61 -> stop at L = 8
    beta, L_stop, levels = oracle.stabilized(None, 0, 1, 0.1, 256, 7)
    assert (beta, L_stop) == (1.61, 8) and sorted(levels) == [1, 2, 4, 8]
    # cap: nothing stabilises before L_max = 4
    beta, L_stop, _ = oracle.stabilized(None, 0, 1, 0.01, 4, 7)
    assert (beta, L_stop) == (1.6, 4)
    # a non-power-of-two cap is reached exactly
    seq.update({3: 100.0})
    beta, L_stop, _ = oracle.stabilized(None, 0, 1, 0.01, 3, 7)
    assert L_stop == 3 and beta == 100.0
    assert oracle.stabilized(None, 5, 5, 0.1, 64, 7)[:2] == (0.0, 1)


def test_rule_is_relative_to_the_longer_level(monkeypatch, oracle_lib):
    """The change is measured against |beta(2L)|, and level L runs on
    level_seed(seed, L): 1.105 vs 1.0 at eps = 0.2 is within 0.1 * 1.105 but
    not within 0.1 * 1.0, so the rule stops at L = 2."""
    seq = {1: 1.0, 2: 1.105, 4: 5.0}
    seen = {}

    def fake_query(g, s, t, eps, L, seed, cfg=None, **kw):
        seen[L] = seed
        return {"beta": seq[L]}

    monkeypatch.setattr(oracle, "query", fake_query)
    beta, L_stop, levels = oracle.stabilized(None, 0, 1, 0.2, 4, 99)
    assert (beta, L_stop) == (1.105, 2) and sorted(levels) == [1, 2]
    assert seen == {L: oracle.level_seed(99, L) for L in (1, 2)}


def test_level_seeds_differ_by_level(oracle_lib):
    seeds = {oracle.level_seed(12345, L) for L in (1, 2, 4, 8, 16)}
    assert len(seeds) == 5
    assert oracle.level_seed(12345, 4) == oracle.level_seed(12345, 4)


def test_stabilized_accuracy_tiny(oracle_lib, tiny_graph):
    g = tiny_graph
    ex = exact.exact_beta_matrix(g.row_ptr, g.col_idx, g.n)
    s, t = uniform_pairs(g.n, 16, 300)
    seeds = query_seeds(16, 301)
    rel = []
    for i in range(16):
        beta, L_stop, _ = oracle.stabilized(g, int(s[i]), int(t[i]), 0.2, 64, int(seeds[i]))
        assert 2 <= L_stop <= 64
        rel.append(abs(beta - ex[s[i], t[i]]) / ex[s[i], t[i]])
    assert np.mean(np.array(rel) <= 0.2) >= 0.9
