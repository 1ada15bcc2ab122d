"""Pins for the oracle's serial walker (Algorithm 1) and its budgets.

* Philox4x32-10 against the published known-answer vectors.
* Neighbour sampling is uniform on N(v) (Algorithm 1 samples X_i uniformly).
* Enumerating every walk of length L <= 4 on small graphs gives
  E[phi_hat | z] = phi(z) = z^T h^(L) (Eq. phi-rw-identity); the walker's
  replicas reproduce it within CLT bounds.
* L = 0 makes every replica equal, so Q_R = phi(z)^2 (Eq. Q-Ustat).
* |U_p| <= 2(L+1)/d_min for every replica (Lemma 3.6).
* With G = 1 the estimator is the plain mean of Q_R, unbiased for beta^(L)
  (Lemmas 3.3 and 3.4).
* THEORY budgets equal the hand-evaluated Eqs. B-value ... K-value.
* PILOT budget reaches the relative-error target of Problem 1 on the tiny graph.
"""

import math
import os

import numpy as np
import pytest

import oracle
from oracle import exact
from pw_inputs import barabasi_albert, complete_graph, er_cycle, query_seeds, uniform_pairs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_philox_known_answers(oracle_lib):
    for row in _read_rows("philox_kat.txt"):
        v = [int(x, 16) for x in row]
        out = oracle.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_neighbour_sampling_uniform(oracle_lib):
    g = barabasi_albert(300, 3, 2)
    v = int(np.argmax(g.degrees))  # a hub: largest neighbour list
    nbrs = g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]
    d = len(nbrs)
    m = 30 * d
    first = np.array([oracle.walk(g, v, 1, 99, w)[1] for w in range(m)])
    counts = np.array([(first == u).sum() for u in nbrs])
    assert counts.sum() == m
    chi2 = ((counts - m / d) ** 2 / (m / d)).sum()
    # chi-square with d-1 dof: mean d-1, sd sqrt(2(d-1))
    assert chi2 < (d - 1) + 6 * math.sqrt(2 * (d - 1))


def test_trajectories_follow_edges(oracle_lib, tiny_graph):
    g = tiny_graph
    adj = set(zip(np.repeat(np.arange(g.n), g.degrees).tolist(), g.col_idx.tolist()))
    for w in range(50):
        tr = oracle.walk(g, 5, 40, 1234, w)
        assert tr[0] == 5
        assert all((int(a), int(b)) in adj for a, b in zip(tr[:-1], tr[1:]))


def _walk_expectation(g, start, L, z):
    """E_start[sum_{i<=L} z_{X_i}/d_{X_i}] by enumerating all walks."""
    deg = g.degrees
    dist = {start: 1.0}
    total = 0.0
    for i in range(L + 1):
        total += sum(p * z[v] / deg[v] for v, p in dist.items())
        if i == L:
            break
        nxt = {}
        for v, p in dist.items():
            for u in g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]:
                nxt[int(u)] = nxt.get(int(u), 0.0) + p / deg[v]
        dist = nxt
    return total


@pytest.mark.parametrize("L", [0, 1, 2, 4])
def test_walk_identity_enumeration(oracle_lib, L):
    g = er_cycle(9, 0.35, 11)
    s, t = 0, 5
    h = exact.series_h(g.row_ptr, g.col_idx, g.n, s, t, L)
    for k in range(4):
        z = oracle.probe_vector(g.n, 2024, k)[0].astype(np.float64)
        phi = float(z @ h)
        enum = _walk_expectation(g, s, L, z) - _walk_expectation(g, t, L, z)
        assert enum == pytest.approx(phi, rel=1e-12, abs=1e-14)


def test_replicas_unbiased_for_phi(oracle_lib):
    g = er_cycle(9, 0.35, 11)
    s, t, L, seed = 0, 5, 4, 2024
    R = 20000
    cfg = oracle.budget_cfg(mode=oracle.MODE_FIXED, B=1, G=1, R=R)
    out = oracle.query(g, s, t, 0.5, L, seed, cfg, want_u=True, want_q=True)
    u = out["u"][0].astype(np.float64)
    z = oracle.probe_vector(g.n, seed, 0)[0].astype(np.float64)
    phi = float(z @ exact.series_h(g.row_ptr, g.col_idx, g.n, s, t, L))
    assert abs(u.mean() - phi) < 5 * u.std() / math.sqrt(R)
    # Q_R is unbiased for phi^2 (Lemma 3.4); its spread is Eq. step1's variance
    var_q = 4 / R * phi**2 * u.var() + 2 / (R * (R - 1)) * u.var() ** 2
    assert abs(out["q"][0] - phi**2) < 6 * math.sqrt(var_q) + 1e-12


def test_L0_replicas_are_deterministic(oracle_lib, tiny_graph):
    g = tiny_graph
    s, t, seed = 4, 90, 77
    cfg = oracle.budget_cfg(mode=oracle.MODE_FIXED, B=3, G=1, R=7)
    out = oracle.query(g, s, t, 0.3, 0, seed, cfg, want_u=True, want_q=True)
    d = g.degrees
    for k in range(3):
        z = oracle.probe_vector(g.n, seed, k)[0]
        u0 = np.float32(np.float32(z[s]) / np.float32(d[s])) - np.float32(np.float32(z[t]) / np.float32(d[t]))
        assert np.all(out["u"][k] == u0)
        assert out["q"][k] == pytest.approx(float(u0) ** 2, rel=1e-12, abs=1e-300)


def test_per_replica_bound_lemma_3_6(oracle_lib, tiny_graph):
    g = tiny_graph
    L = 32
    cfg = oracle.budget_cfg(mode=oracle.MODE_FIXED, B=20, G=1, R=64)
    out = oracle.query(g, 10, 20, 0.2, L, 5, cfg, want_u=True)
    assert np.abs(out["u"]).max() <= 2 * (L + 1) / g.d_min


def test_mean_of_estimates_is_unbiased(oracle_lib):
    g = barabasi_albert(60, 2, 7)
    s, t, L = 3, 40, 6
    want = exact.series_beta(g.row_ptr, g.col_idx, g.n, s, t, L)
    cfg = oracle.budget_cfg(mode=oracle.MODE_FIXED, B=40, G=1, R=8)
    seeds = query_seeds(300, 3)
    beta, _, st = oracle.query_many(g, np.full(300, s), np.full(300, t), 0.5, L, seeds, cfg)
    assert np.all(st == 0)
    assert abs(beta.mean() - want) < 5 * beta.std() / math.sqrt(beta.size)


def test_visits_are_the_walks_of_every_replica(oracle_lib, tiny_graph):
    """Replica p of probe k runs walk 2(kR + p) from s and walk 2(kR + p) + 1
    from t (reading 8), each of L transitions with X_0 counted (L + 1 visits,
    Algorithm 1's inner loop): the query's visit counts equal the histogram of
    those trajectories drawn one by one."""
    g = tiny_graph
    s, t, L, seed = 3, 77, 7, 4242
    B, G, R = 2, 3, 8
    cfg = oracle.budget_cfg(mode=oracle.MODE_FIXED, B=B, G=G, R=R)
    out = oracle.query(g, s, t, 0.2, L, seed, cfg, want_visits=True)
    K = B * G
    assert int(out["visits"].sum()) == 2 * K * R * (L + 1)
    want = np.zeros(g.n, np.int64)
    for k in range(K):
        for p in range(R):
            for side, start in ((0, s), (1, t)):
                traj = oracle.walk(g, start, L, seed, 2 * (k * R + p) + side, oracle.TAG_WALK)
                assert len(traj) == L + 1 and traj[0] == start
                np.add.at(want, traj, 1)
    np.testing.assert_array_equal(out["visits"].astype(np.int64), want)


def test_theory_budget_golden(oracle_lib):
    for row in _read_rows("budget_theory.txt"):
        assert row[0].startswith("K")
        g = complete_graph(int(row[0][1:]))
        eps, delta, L, s, t = float(row[1]), float(row[2]), int(row[3]), int(row[4]), int(row[5])
        B, G, K, R = (int(x) for x in row[6:10])
        got = oracle.budget(g, s, t, eps, L, 1, oracle.budget_cfg(mode=oracle.MODE_THEORY, delta=delta))
        assert (got["B"], got["G"], got["K"], got["R"]) == (B, G, K, R)


def test_scaled_and_fixed_budgets(oracle_lib):
    g = complete_graph(10)
    got = oracle.budget(g, 0, 1, 0.1, 4, 1, oracle.budget_cfg(mode=oracle.MODE_SCALED, c_B=0.01, c_R=0.1, R_max=64))
    assert got["B"] == 448 and got["G"] == 37 and got["R"] == 64  # ceil(84.2) clamped to R_max
    got = oracle.budget(g, 0, 1, 0.1, 4, 1, oracle.budget_cfg(mode=oracle.MODE_FIXED, B=3, G=5, R=9))
    assert (got["B"], got["G"], got["K"], got["R"]) == (3, 5, 15, 9)


def test_pilot_budget_shape(oracle_lib, tiny_graph):
    got = oracle.budget(tiny_graph, 3, 77, 0.2, 32, 12345)
    assert got["B"] == 13 and got["G"] == 37 and got["K"] == 481  # ceil(0.5 / 0.2^2) = 13
    assert got["R"] % 32 == 0 and 32 <= got["R"] <= 4096
    d = tiny_graph.degrees
    theta0 = 0.125 * (1 - 0.1) * (1 / d[3] + 1 / d[77]) ** 2
    assert got["theta_hat"] >= theta0
    assert got["R"] >= 4 * got["sigma2_hat"] / got["theta_hat"]


def test_same_node_and_bad_arguments(oracle_lib, tiny_graph):
    assert oracle.query(tiny_graph, 7, 7, 0.2, 32, 1)["beta"] == 0.0
    for args in ((0, 1, 0.0, 32), (0, 1, 1.0, 32), (0, 200, 0.2, 32), (-1, 1, 0.2, 32), (0, 1, 0.2, -1)):
        with pytest.raises(ValueError):
            oracle.query(tiny_graph, args[0], args[1], args[2], args[3], 1)


def test_default_seed_depends_on_query(oracle_lib):
    a = oracle.default_seed(1, 3, 4, 0.1, 200)
    assert a == oracle.default_seed(1, 3, 4, 0.1, 200)
    others = {oracle.default_seed(1, 4, 3, 0.1, 200), oracle.default_seed(2, 3, 4, 0.1, 200),
              oracle.default_seed(1, 3, 4, 0.2, 200), oracle.default_seed(1, 3, 4, 0.1, 201)}
    assert a not in others and len(others) == 4


def test_pilot_accuracy_problem_1(oracle_lib, tiny_graph):
    """>= 95% of queries within eps of the exact beta (Problem 1, Theorem 3.8's target)."""
    g = tiny_graph
    ex = exact.exact_beta_matrix(g.row_ptr, g.col_idx, g.n)
    s, t = uniform_pairs(g.n, 32, 100)
    seeds = query_seeds(32, 200)
    beta, _, st = oracle.query_many(g, s, t, 0.2, 32, seeds)
    assert np.all(st == 0)
    rel = np.abs(beta - ex[s, t]) / ex[s, t]
    assert (rel <= 0.2).mean() >= 0.95


def _median_rows():
    rows = []
    with open(os.path.join(GOLDEN, "median_of_means.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            head, vals = line.split("|")
            B, G, res = head.split()
            rows.append((int(B), int(G), float(res), [float(x) for x in vals.split()]))
    return rows


def test_median_of_means_golden(oracle_lib):
    """Hand-evaluated medians of contiguous block means, odd and even G
    (Eq. final-estimator; an even G takes the mean of the two middle means)."""
    rows = _median_rows()
    assert any(G % 2 == 0 for _, G, _, _ in rows) and any(G % 2 == 1 for _, G, _, _ in rows)
    for B, G, res, q in rows:
        assert oracle.median_of_means(q, B, G) == res, (B, G, q)


def test_even_G_query_takes_middle_pair(oracle_lib, tiny_graph):
    """A FIXED budget with G = 4: beta_hat is numpy's median of the query's own
    four block means (mean of the two middle ones), not either middle value."""
    cfg = oracle.budget_cfg(mode=oracle.MODE_FIXED, B=5, G=4, R=16)
    out = oracle.query(tiny_graph, 11, 150, 0.2, 16, 4321, cfg, want_q=True)
    means = out["q"].reshape(4, 5).mean(axis=1)
    srt = np.sort(means)
    assert srt[1] != srt[2]
    assert out["beta"] == pytest.approx(float(np.median(means)), rel=1e-14, abs=1e-300)


def test_G_for_even_deltas(oracle_lib, tiny_graph):
    """G = ceil(8 ln(1/delta)) (Eq. G-value): 24 at delta = 0.05 (8 ln 20 = 23.97)
    and 32 at delta = 0.02 (8 ln 50 = 31.30), both even."""
    for delta, G in ((0.05, 24), (0.02, 32), (0.01, 37)):
        got = oracle.budget(tiny_graph, 3, 77, 0.2, 32, 1, oracle.budget_cfg(delta=delta))
        assert got["G"] == G and got["K"] == 13 * G


def _hub_graph():
    return barabasi_albert(3000, 2, 5)


@pytest.mark.parametrize("s,t,L,seed,eps", [(3, 77, 32, 12345, 0.2), (10, 190, 8, 99, 0.1), (0, 1, 0, 5, 0.3),
                                            (42, 43, 20, 2**63 + 9, 0.05), ("hub", 0, 32, 2, 0.2)])
def test_pilot_statistics_from_replicas(oracle_lib, tiny_graph, s, t, L, seed, eps):
    """PILOT's estimates from the pilot replicas themselves (Lemma 3.7's
    sufficient condition R >= 4 sigma^2 / theta):
      sigma2_hat = mean over pilot probes of numpy's unbiased sample variance;
      q_bar      = mean of the probes' U-statistics, written as mean^2 - var/R0
                   (equal to Eq. Q-Ustat by S1^2 - S2 = R(R-1) mean^2 - (R-1) var);
      theta_hat  = max(q_bar, theta_0), theta_0 = (1/8)(1 - eps/2)(1/d_s + 1/d_t)^2;
      R          = 4 sigma2_hat / theta_hat rounded up to whole warps of 32, in [32, 4096].
    The "hub" case (the two largest hubs of a 3000-node BA graph) has a negative
    pilot mean, so the theta_0 floor and the R clamp decide its budget."""
    g = tiny_graph
    if s == "hub":
        g, s = _hub_graph(), 1
    u = oracle.pilot_u(g, s, t, L, seed).astype(np.float64)
    K0, R0 = u.shape
    assert (K0, R0) == (64, 32)
    mean = u.mean(axis=1)
    var = u.var(axis=1, ddof=1)
    sigma2 = float(var.mean())
    q_bar = float((mean**2 - var / R0).mean())
    scale = float((mean**2 + var / R0).mean())  # size of the terms that cancel in q
    d = g.degrees
    theta0 = 0.125 * (1 - eps / 2) * (1 / d[s] + 1 / d[t]) ** 2
    got = oracle.budget(g, s, t, eps, L, seed)
    assert got["sigma2_hat"] == pytest.approx(sigma2, rel=1e-12, abs=1e-300)
    assert abs(got["q_bar"] - q_bar) <= 1e-12 * scale + 1e-300
    assert got["theta_hat"] == pytest.approx(max(q_bar, theta0), rel=1e-9, abs=1e-12 * scale)
    r = 4 * sigma2 / got["theta_hat"]
    lo = min(4096, max(32, 32 * math.ceil(math.ceil(r * (1 - 1e-9)) / 32)))
    hi = min(4096, max(32, 32 * math.ceil(math.ceil(r * (1 + 1e-9)) / 32)))
    assert lo <= got["R"] <= hi


def _fraction_sum(vals):
    from fractions import Fraction

    return float(sum((Fraction(float(v)) for v in vals), Fraction(0)))


def test_exact_sums_are_correctly_rounded(oracle_lib):
    """S1 = sum U_p and S2 = sum U_p^2 are the exact sums rounded once (round to
    nearest, ties to even): equal to math.fsum and to exact rational arithmetic
    on FP32 values spread over 40 binades with heavy cancellation, whatever
    their order."""
    rng = np.random.default_rng(17)
    for trial in range(20):
        n = int(rng.integers(1, 3000))
        mag = 2.0 ** rng.integers(-30, 10, size=n)
        u = (rng.standard_normal(n) * mag).astype(np.float32)
        if trial % 3 == 0:  # cancellation: add the negatives of most values back
            u = np.concatenate([u, -u[: n // 2 + 1]]).astype(np.float32)
        x = u.astype(np.float64)
        s1, s2 = oracle.exact_sum_f32(u), oracle.exact_sum_f32(u, square=True)
        assert s1 == math.fsum(x.tolist()) == _fraction_sum(x)
        assert s2 == math.fsum((x * x).tolist()) == _fraction_sum(x * x)
        perm = rng.permutation(u.size)
        assert oracle.exact_sum_f32(u[perm]) == s1 and oracle.exact_sum_f32(u[perm], square=True) == s2


def test_exact_sum_ties_and_edges(oracle_lib):
    e = 2.0**-53
    cases = [
        ([1.0, e], 1.0),                       # exact tie, even neighbour below
        ([1.0, 2 * e, e], 1.0 + 4 * e),        # 1 + 3e: tie, even neighbour above
        ([1.0, e, 2.0**-80], 1.0 + 2 * e),     # just above the tie
        ([1.0, e, e], 1.0 + 2 * e),            # no tie at all: sequential FP64 would give 1.0
        ([e, e, 1.0], 1.0 + 2 * e),
        ([-1.0, -e, -e], -(1.0 + 2 * e)),
        ([3.0, -3.0], 0.0),
        ([], 0.0),
        ([2.0**100, 1.0, -(2.0**100)], 1.0),
    ]
    for vals, want in cases:
        u = np.array(vals, np.float32)
        assert u.astype(np.float64).tolist() == vals
        got = oracle.exact_sum_f32(u)
        assert got == want and math.copysign(1.0, got) == math.copysign(1.0, want), (vals, got, want)


@pytest.mark.parametrize("cap", [1.0, 2.0])
@pytest.mark.parametrize("s,t,eps,L,seed", [(3, 77, 0.2, 32, 12345), (10, 190, 0.1, 8, 99), (42, 43, 0.15, 20, 7),
                                            ("hub", 0, 0.2, 32, 2)])
def test_adaptive_budget_stopping_rule(oracle_lib, tiny_graph, s, t, eps, L, seed, cap):
    """ADAPTIVE budget: from the first stage's G ceil(B/4) values of Q_R
    (B: PILOT's), B* = ceil((pi/2) z^2 s^2 / (G eps^2 theta^2)) clamped to
    [ceil(B/4), cap B] (numpy's unbiased variance and mean, theta =
    max(mean, theta_0)); the estimate is numpy's median of the G block means
    of the first G B* probes, which extend the PILOT query's own probes."""
    g = tiny_graph
    if s == "hub":
        g, s = _hub_graph(), 1
    z = 2.2
    cfg = oracle.budget_cfg(mode=oracle.MODE_ADAPTIVE, z=z, cap=cap)
    out = oracle.query(g, s, t, eps, L, seed, cfg, want_q=True)
    pilot = oracle.query(g, s, t, eps, L, seed, oracle.budget_cfg(), want_q=True)
    assert out["R"] == pilot["R"] and out["G"] == pilot["G"]
    Bp, G = pilot["B"], pilot["G"]
    B1 = -(-Bp // 4)
    q1 = out["q"][: G * B1]
    d = g.degrees
    theta0 = 0.125 * (1 - eps / 2) * (1 / d[s] + 1 / d[t]) ** 2
    theta = max(q1.mean(), theta0)
    x = math.pi / 2 * z * z * q1.var(ddof=1) / (G * eps * eps * theta * theta)
    Bcap = math.ceil(cap * Bp - 1e-9)
    lo = min(Bcap, max(B1, math.ceil(x * (1 - 1e-9))))
    hi = min(Bcap, max(B1, math.ceil(x * (1 + 1e-9))))
    assert lo <= out["B"] <= hi and out["K"] == G * out["B"]
    common = min(out["K"], pilot["K"])
    np.testing.assert_array_equal(out["q"][:common], pilot["q"][:common])  # the same probes, extended
    means = out["q"].reshape(G, out["B"]).mean(axis=1)
    assert out["beta"] == pytest.approx(float(np.median(means)), rel=1e-12, abs=1e-300)


def test_adaptive_rule_golden(oracle_lib):
    """Hand-evaluated stopping rule (tests/golden/adaptive_B.txt): the unbiased
    variance, the (pi/2) z^2 factor, the theta_0 floor and both clamps."""
    n_rows = 0
    with open(os.path.join(GOLDEN, "adaptive_B.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            head, vals = line.split("|")
            B1, B, G, eps, z, ds, dt, want = head.split()
            q = [float(x) for x in vals.split()]
            got = oracle.adaptive_B(q, int(B1), int(B), int(G), float(eps), float(z), float(ds), float(dt))
            assert got == int(want), (line, got)
            n_rows += 1
    assert n_rows == 6
