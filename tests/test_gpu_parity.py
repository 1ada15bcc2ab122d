"""GPU parity: the CUDA path through the C ABI against the oracle.

Integer work is compared bit for bit (Philox words, probe vectors, walk
trajectories, visit counts).  Floating point: U_p (FP32, fixed step order)
is bit-exact; Q_R and beta_hat use FP64 sums in the oracle's order, so they
are bit-exact too; every comparison also states the required tolerance of
1e-5 relative, which is the bar."""

import math
import os

import numpy as np
import pytest

import oracle
from oracle import exact
from pw_inputs import (barabasi_albert, complete_graph, cycle_graph, er_cycle, eps_uniform, from_edges, path_graph,
                       query_seeds, uniform_pairs)

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def pw():
    from paper_2512_05460_gb300 import build

    build.build()
    from paper_2512_05460_gb300 import probewalk

    probewalk.lib()
    return probewalk


@pytest.fixture(scope="module")
def tiny(pw, tiny_graph):
    g = pw.Graph(tiny_graph.row_ptr, tiny_graph.col_idx)
    yield tiny_graph, g
    g.close()


@pytest.fixture(scope="module")
def ba_graph():
    return barabasi_albert(100_000, 5, 1)


@pytest.fixture(scope="module")
def ba(pw, ba_graph):
    g = pw.Graph(ba_graph.row_ptr, ba_graph.col_idx)
    yield ba_graph, g
    g.close()


def test_graph_info(pw, tiny):
    host, g = tiny
    info = pw.pw_graph_info(g.handle)
    assert info["n"] == host.n and info["nnz"] == host.nnz
    assert info["d_min"] == host.d_min and info["d_max"] == host.d_max
    assert info["bipartite"] == host.is_bipartite()


def test_philox_known_answers_on_device(pw, tiny):
    _, g = tiny
    with open(os.path.join(GOLDEN, "philox_kat.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for row in rows:
        v = [int(x, 16) for x in row]
        assert [int(x) for x in pw.pw_debug_philox(g.handle, v[0:4], v[4:6])] == v[6:10]


@pytest.mark.parametrize("graph_fn", [lambda: er_cycle(200, 8 / 199, 0), lambda: complete_graph(7),
                                      lambda: cycle_graph(16), lambda: barabasi_albert(3000, 3, 5)])
def test_probe_vectors_bit_exact(pw, oracle_lib, graph_fn):
    host = graph_fn()
    with pw.Graph(host.row_ptr, host.col_idx) as g:
        for seed in (1, 2**64 - 3, 987654321):
            for k in (0, 1, 77, 2**31 + 5):
                for tag in (pw.TAG_PROBE, pw.TAG_PROBE_PILOT):
                    z_dev, r_dev = pw.pw_debug_probe(g.handle, host.n, seed, k, tag)
                    z_orc, _, r_orc = oracle.probe_vector(host.n, seed, k, tag)
                    assert r_dev == r_orc
                    np.testing.assert_array_equal(z_dev, z_orc)


def test_trajectories_bit_exact(pw, oracle_lib, tiny):
    host, g = tiny
    rng = np.random.default_rng(0)
    for _ in range(40):
        start = int(rng.integers(host.n))
        L = int(rng.integers(0, 70))
        seed = int(rng.integers(0, 2**63))
        wid = int(rng.integers(0, 2**40))
        tag = int(rng.choice([pw.TAG_WALK, pw.TAG_WALK_PILOT]))
        np.testing.assert_array_equal(pw.pw_debug_walk(g.handle, start, L, seed, wid, tag),
                                      oracle.walk(host, start, L, seed, wid, tag))


def test_device_exact_sums_match_oracle(pw, oracle_lib, tiny):
    """The walk kernels' per-probe accumulator (exact integer digits, one
    rounding) gives the oracle's S1 and S2 bit for bit, ties and near-ties
    included, on values in the range every replica value lies in."""
    _, g = tiny
    e = 2.0**-53
    cases = [[1.0, e], [1.0, 2 * e, e], [1.0, e, e], [e, e, 1.0], [-1.0, -e, -e], [3.0, -3.0], [],
             [2.0**20, 2.0**-33, 2.0**-54], [2.0**20, 2.0**-33], [2.0**32, -1.0, 2.0**-54]]
    for vals in cases:
        u = np.array(vals, np.float32)
        got = pw.pw_debug_exact_sum(g.handle, u)
        want = (oracle.exact_sum_f32(u), oracle.exact_sum_f32(u, square=True))
        assert got == want, (vals, got, want)
    rng = np.random.default_rng(23)
    for trial in range(12):
        n = int(rng.integers(1, 5000))
        u = (rng.standard_normal(n) * 2.0 ** rng.integers(-25, 12, size=n)).astype(np.float32)
        if trial % 2:
            u = np.concatenate([u, -u[: n // 2]])
        got = pw.pw_debug_exact_sum(g.handle, u)
        assert got == (oracle.exact_sum_f32(u), oracle.exact_sum_f32(u, square=True))


def test_mixed_walk_kernels_in_one_batch(pw, oracle_lib, tiny):
    """The walk kernel is chosen per query on the device: with L = 0 the table
    does not pay (2 R visits per probe against n Feistel passes), with longer
    walks it does, so one batch runs both kernels; every estimate equals the
    oracle's and the forced single-kernel runs'."""
    host, g = tiny
    s, t = uniform_pairs(host.n, 20, 420)
    seeds = query_seeds(20, 421)
    L = np.where(np.arange(20) % 2 == 0, 0, 24).astype(np.int32)
    pw.pw_profile(g.handle, enable=True, reset=True)
    auto, st = pw.pw_query_batch(g.handle, s, t, 0.25, L, seeds)
    assert pw.pw_profile(g.handle, enable=False, reset=True)["walk_mode"] == 3
    assert np.all(st == 0)
    want, _, ost = oracle.query_many(host, s, t, 0.25, L, seeds)
    np.testing.assert_allclose(auto, want, rtol=REL_TOL, atol=0)
    np.testing.assert_array_equal(auto, want)
    for mode in (1, 2):
        forced, _ = pw.pw_query_batch(g.handle, s, t, 0.25, L, seeds, pw.make_params(walk_mode=mode))
        np.testing.assert_array_equal(forced, want)


@pytest.mark.parametrize("graph_fn", [lambda: er_cycle(200, 8 / 199, 0), lambda: barabasi_albert(3000, 3, 5)])
def test_layouts_give_the_same_walks(pw, oracle_lib, graph_fn):
    """Fused records (one 16-byte gather per step) and col_idx plus node
    records (two gathers) give the same trajectories and the same estimates,
    in both walk kernels and the server."""
    host = graph_fn()
    s, t = uniform_pairs(host.n, 8, 440)
    seeds = query_seeds(8, 441)
    want, _, _ = oracle.query_many(host, s, t, 0.25, 20, seeds)
    for flags, layout in ((pw.LOAD_FUSED, 1), (pw.LOAD_SPLIT, 2)):
        with pw.Graph(host.row_ptr, host.col_idx, flags=flags) as g:
            assert pw.pw_profile(g.handle, enable=False)["layout"] == layout
            for w in range(5):
                np.testing.assert_array_equal(pw.pw_debug_walk(g.handle, int(s[w]), 30, 99, w),
                                              oracle.walk(host, int(s[w]), 30, 99, w))
            for mode in (1, 2):
                b, st = pw.pw_query_batch(g.handle, s, t, 0.25, 20, seeds, pw.make_params(walk_mode=mode))
                assert np.all(st == 0)
                np.testing.assert_array_equal(b, want)
            srv = pw.pw_server_create(g.handle, None, 1 << 24)
            try:
                tk = [pw.pw_server_submit(srv, int(s[i]), int(t[i]), 0.25, 20, int(seeds[i])) for i in range(8)]
                pw.pw_server_drain(srv, 60000)
                got = [pw.pw_server_poll(srv, x)[1] for x in tk]
            finally:
                pw.pw_server_destroy(srv)
            np.testing.assert_array_equal(got, want)
            ok = pw.pw_series_batch(g.handle, s, t, np.full(8, 20, np.int32))
            np.testing.assert_allclose(ok, exact.series_beta_many(host.row_ptr, host.col_idx, host.n, s, t, 20),
                                       rtol=1e-9, atol=0)


def test_repeated_calls_replay_a_cuda_graph(pw, oracle_lib, tiny):
    """A host-array call runs eagerly the first time its shape is seen, is
    captured as a CUDA graph the second time and replayed afterwards: every
    call gives the oracle's estimates and counts the same kernel launches."""
    host, g = tiny
    s, t = uniform_pairs(host.n, 6, 430)
    seeds = query_seeds(6, 431)
    want, _, _ = oracle.query_many(host, s, t, 0.2, 32, seeds)
    counts = []
    for i in range(6):
        pw.pw_launch_count(reset=True)
        assert pw.pw_query(g.handle, int(s[i]), int(t[i]), 0.2, 32, int(seeds[i])) == want[i]
        counts.append(pw.pw_launch_count(reset=True))
    assert len(set(counts)) == 1 and counts[0] > 0
    for _ in range(3):
        b, st = pw.pw_query_batch(g.handle, s, t, 0.2, 32, seeds)
        assert np.all(st == 0)
        np.testing.assert_array_equal(b, want)
    b, _ = pw.pw_query_batch(g.handle, s[:4], t[:4], 0.2, 32, seeds[:4])  # another shape
    np.testing.assert_array_equal(b, want[:4])
    b, _ = pw.pw_query_batch(g.handle, s, t, 0.2, 32, seeds)
    np.testing.assert_array_equal(b, want)


def _compare_query(pw, host, g, s, t, eps, L, seed, params, cfg):
    dev = pw.pw_debug_query(g.handle, host.n, s, t, eps, L, seed, params, q_cap=1 << 22, u_cap=1 << 26,
                            want_visits=True)
    orc = oracle.query(host, s, t, eps, L, seed, cfg, want_q=True, want_u=True, want_visits=True)
    assert (dev["B"], dev["G"], dev["K"], dev["R"]) == (orc["B"], orc["G"], orc["K"], orc["R"])
    assert dev["sigma2_hat"] == orc["sigma2_hat"] and dev["q_bar"] == orc["q_bar"]
    np.testing.assert_array_equal(dev["u"], orc["u"])          # every U_p, bit for bit
    np.testing.assert_array_equal(dev["visits"], orc["visits"])  # visit counts
    np.testing.assert_array_equal(dev["q"], orc["q"])
    assert dev["beta"] == orc["beta"]
    assert abs(dev["beta"] - orc["beta"]) <= REL_TOL * abs(orc["beta"])
    return dev, orc


@pytest.mark.parametrize("walk_mode", [1, 2])
def test_debug_query_pilot_bit_exact(pw, oracle_lib, tiny, walk_mode):
    host, g = tiny
    params = pw.make_params(walk_mode=walk_mode)
    for s, t, seed in ((3, 77, 12345), (0, 199, 1), (150, 9, 2**62 + 11)):
        _compare_query(pw, host, g, s, t, 0.2, 32, seed, params, oracle.budget_cfg())


@pytest.mark.parametrize("walk_mode", [1, 2])
@pytest.mark.parametrize("B,G,R,L", [(3, 1, 2, 0), (5, 3, 7, 1), (4, 5, 45, 13), (2, 3, 70, 33), (1, 1, 33, 4)])
def test_debug_query_fixed_ragged_bit_exact(pw, oracle_lib, tiny, B, G, R, L, walk_mode):
    host, g = tiny
    params = pw.make_params(budget_mode=pw.PW_BUDGET_FIXED, B=B, G=G, R=R, walk_mode=walk_mode)
    cfg = oracle.budget_cfg(mode=oracle.MODE_FIXED, B=B, G=G, R=R)
    _compare_query(pw, host, g, 10, 20, 0.3, L, 424242, params, cfg)


@pytest.mark.parametrize("walk_mode", [1, 2])
def test_even_G_delta_005_bit_exact(pw, oracle_lib, tiny, walk_mode):
    """delta = 0.05 gives G = 24 block means, an even count: the median is the
    mean of the two middle ones on the device as in the oracle (pw_debug_query,
    pw_query_batch and pw_query, element by element)."""
    host, g = tiny
    params = pw.make_params(delta=0.05, walk_mode=walk_mode)
    cfg = oracle.budget_cfg(delta=0.05)
    dev, _ = _compare_query(pw, host, g, 3, 77, 0.2, 32, 12345, params, cfg)
    assert dev["G"] == 24
    s, t = uniform_pairs(host.n, 16, 410)
    seeds = query_seeds(16, 411)
    beta, st = pw.pw_query_batch(g.handle, s, t, 0.2, 32, seeds, params)
    ob, ob_budget, ost = oracle.query_many(host, s, t, 0.2, 32, seeds, cfg)
    assert np.all(st == 0) and np.all(ost == 0) and np.all(ob_budget[:, 1] == 24)
    np.testing.assert_allclose(beta, ob, rtol=REL_TOL, atol=0)
    np.testing.assert_array_equal(beta, ob)
    for i in range(3):
        assert pw.pw_query(g.handle, int(s[i]), int(t[i]), 0.2, 32, int(seeds[i]), params) == ob[i]
    # delta = 0.02 gives G = 32
    b2, _ = pw.pw_query_batch(g.handle, s[:4], t[:4], 0.2, 32, seeds[:4], pw.make_params(delta=0.02))
    o2, bud2, _ = oracle.query_many(host, s[:4], t[:4], 0.2, 32, seeds[:4], oracle.budget_cfg(delta=0.02))
    assert np.all(bud2[:, 1] == 32)
    np.testing.assert_array_equal(b2, o2)


@pytest.mark.parametrize("walk_mode", [1, 2])
def test_adaptive_budget_bit_exact(pw, oracle_lib, tiny, walk_mode):
    """ADAPTIVE budget (first stage, stopping rule, second stage): the stopping
    B*, every U_p of both stages, every Q_R, the visit counts and the estimate
    equal the oracle's; a batch of 24 mixed queries equals the oracle query by
    query, and the queries' B differ from PILOT's (up to twice it)."""
    host, g = tiny
    params = pw.make_params(budget_mode=pw.PW_BUDGET_ADAPTIVE, walk_mode=walk_mode)
    cfg = oracle.budget_cfg(mode=oracle.MODE_ADAPTIVE)
    for s, t, seed in ((3, 77, 12345), (0, 199, 1), (150, 9, 2**62 + 11)):
        _compare_query(pw, host, g, s, t, 0.2, 32, seed, params, cfg)
    s, t = uniform_pairs(host.n, 24, 450)
    eps = eps_uniform(24, 0.1, 0.3, 451)
    L = np.random.default_rng(452).integers(0, 40, size=24).astype(np.int32)
    seeds = query_seeds(24, 453)
    beta, st = pw.pw_query_batch(g.handle, s, t, eps, L, seeds, params)
    want, budgets, ost = oracle.query_many(host, s, t, eps, L, seeds, cfg)
    assert np.all(st == 0) and np.all(ost == 0)
    np.testing.assert_allclose(beta, want, rtol=REL_TOL, atol=0)
    np.testing.assert_array_equal(beta, want)
    _, pilot_budgets, _ = oracle.query_many(host, s, t, eps, L, seeds)
    assert np.all(budgets[:, 0] <= 2 * pilot_budgets[:, 0]) and np.any(budgets[:, 0] != pilot_budgets[:, 0])
    for i in range(3):
        assert pw.pw_query(g.handle, int(s[i]), int(t[i]), float(eps[i]), int(L[i]), int(seeds[i]), params) == want[i]


@pytest.mark.parametrize("mode", ["THEORY", "SCALED"])
def test_budget_modes_match_oracle(pw, oracle_lib, tiny, mode):
    host, g = tiny
    if mode == "THEORY":
        params = pw.make_params(budget_mode=pw.PW_BUDGET_THEORY)
        cfg = oracle.budget_cfg(mode=oracle.MODE_THEORY)
    else:
        params = pw.make_params(budget_mode=pw.PW_BUDGET_SCALED, c_B=0.001, c_R=0.01, R_max=500)
        cfg = oracle.budget_cfg(mode=oracle.MODE_SCALED, c_B=0.001, c_R=0.01, R_max=500)
    for s, t, eps, L in ((1, 2, 0.5, 4), (5, 100, 0.1, 32), (7, 8, 0.05, 0)):
        dev = pw.pw_budget(g.handle, s, t, eps, L, 99, params)
        orc = oracle.budget(host, s, t, eps, L, 99, cfg)
        assert (dev["B"], dev["G"], dev["K"], dev["R"]) == (orc["B"], orc["G"], orc["K"], orc["R"])


@pytest.mark.parametrize("walk_mode", [0, 1, 2])
def test_tiny_batch_parity_and_accuracy(pw, oracle_lib, tiny, walk_mode):
    """64 queries of the tiny workload: per-query beta_hat equal to the oracle
    (tolerance 1e-5 rel; in fact bit-exact) and >= 95% within eps of the exact beta."""
    host, g = tiny
    s, t = uniform_pairs(host.n, 64, 100)
    seeds = query_seeds(64, 200)
    beta, st = pw.pw_query_batch(g.handle, s, t, 0.2, 32, seeds, pw.make_params(walk_mode=walk_mode))
    assert np.all(st == 0)
    ob, _, ost = oracle.query_many(host, s, t, 0.2, 32, seeds)
    assert np.all(ost == 0)
    np.testing.assert_allclose(beta, ob, rtol=REL_TOL, atol=0)
    assert np.array_equal(beta, ob)
    ex = exact.exact_beta_matrix(host.row_ptr, host.col_idx, host.n)[s, t]
    assert (np.abs(beta - ex) / ex <= 0.2).mean() >= 0.95


def test_alone_equals_in_mix(pw, tiny):
    host, g = tiny
    s, t = uniform_pairs(host.n, 24, 5)
    eps = eps_uniform(24, 0.15, 0.4, 6)
    L = np.random.default_rng(7).integers(0, 40, size=24).astype(np.int32)
    seeds = query_seeds(24, 8)
    mix, st = pw.pw_query_batch(g.handle, s, t, eps, L, seeds)
    assert np.all(st == 0)
    for i in range(24):
        alone = pw.pw_query(g.handle, int(s[i]), int(t[i]), float(eps[i]), int(L[i]), int(seeds[i]))
        assert alone == mix[i]
    # reversed order inside the batch
    rev, _ = pw.pw_query_batch(g.handle, s[::-1], t[::-1], eps[::-1], L[::-1], seeds[::-1])
    np.testing.assert_array_equal(rev[::-1], mix)


def test_edge_cases(pw, oracle_lib, tiny):
    host, g = tiny
    # empty batch
    b, st = pw.pw_query_batch(g.handle, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    assert b.size == 0
    # s == t gives exactly 0 without walks; invalid queries get a per-query status
    s = np.array([5, 5, -1, 3, 3, 4])
    t = np.array([5, 6, 2, 200, 7, 9])
    eps = np.array([0.2, 0.2, 0.2, 0.2, 1.5, 0.2])
    L = np.array([32, 32, 32, 32, 32, -3])
    beta, st = pw.pw_query_batch(g.handle, s, t, eps, L, query_seeds(6, 1))
    assert beta[0] == 0.0 and st[0] == 0
    assert st[1] == 0 and np.isfinite(beta[1])
    assert list(st[2:]) == [pw.PW_ERR_ARG] * 4
    assert np.all(np.isnan(beta[2:]))
    assert pw.pw_query(g.handle, 9, 9, 0.2, 32) == 0.0
    for bad in ((0, 200, 0.2, 32), (0, 1, 0.0, 32), (0, 1, 1.0, 32), (0, 1, 0.2, -1)):
        with pytest.raises(pw.PWError):
            pw.pw_query(g.handle, *bad)
    # default seeds: library and oracle agree on the seed, hence on the estimate
    params = pw.make_params(seed=777, budget_mode=pw.PW_BUDGET_FIXED, B=2, G=1, R=5)
    got = pw.pw_query(g.handle, 1, 2, 0.3, 6, None, params)
    want = oracle.query(host, 1, 2, 0.3, 6, oracle.default_seed(777, 1, 2, 0.3, 6),
                        oracle.budget_cfg(mode=oracle.MODE_FIXED, B=2, G=1, R=5))["beta"]
    assert got == want


def test_invalid_graphs_rejected(pw):
    rp = np.array([0, 1, 2, 3])
    with pytest.raises(pw.PWError):  # asymmetric
        pw.pw_graph_load(rp, np.array([1, 2, 0]))
    with pytest.raises(pw.PWError):  # disconnected: two edges 0-1, 2-3
        pw.pw_graph_load(np.array([0, 1, 2, 3, 4]), np.array([1, 0, 3, 2]))
    with pytest.raises(pw.PWError):  # isolated node 2
        pw.pw_graph_load(np.array([0, 1, 2, 2]), np.array([1, 0]))
    with pytest.raises(pw.PWError):  # self-loop
        pw.pw_graph_load(np.array([0, 2, 3]), np.array([0, 1, 0]))


def test_bipartite_flag(pw):
    p = path_graph(6)
    with pw.Graph(p.row_ptr, p.col_idx) as g:
        assert g.info["bipartite"]


def test_device_api_matches_host_api(pw, tiny):
    torch = pytest.importorskip("torch")
    host, g = tiny
    s, t = uniform_pairs(host.n, 40, 11)
    seeds = query_seeds(40, 12)
    eps = np.full(40, 0.25)
    L = np.full(40, 20, np.int32)
    want, _ = pw.pw_query_batch(g.handle, s, t, eps, L, seeds)
    dev = torch.device("cuda:0")
    ds, dt = torch.from_numpy(s).to(dev), torch.from_numpy(t).to(dev)
    de, dl = torch.from_numpy(eps).to(dev), torch.from_numpy(L).to(dev)
    dseed = torch.from_numpy(seeds.view(np.int64)).to(dev)
    beta = torch.empty(40, dtype=torch.float64, device=dev)
    status = torch.empty(40, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pw.pw_query_batch_device(g.handle, 40, ds, dt, de, dl, dseed, beta, status, stream=stream)
    stream.synchronize()
    np.testing.assert_array_equal(beta.cpu().numpy(), want)
    assert int(status.abs().sum()) == 0


# ---------------------------------------------------------------------------
# Full-size BA workload (n = 100,000, m = 5; 1,000 queries; L = 200; eps = 0.1)
# in the bench's launch configuration.  The oracle recomputes sampled probes
# one by one, and two whole queries.
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def ba_batch(pw, ba):
    host, g = ba
    s, t = uniform_pairs(host.n, 1000, 101)
    seeds = query_seeds(1000, 1001)
    rng = np.random.default_rng(3)
    sel_q = rng.integers(0, 1000, size=24)
    # probe indices are drawn below K for every query (K = 37 * ceil(0.5 / 0.1^2) = 1850)
    sel_k = rng.integers(0, 1850, size=24)
    beta, st, KR, qsel = pw.pw_debug_batch_probe_q(g.handle, s, t, 0.1, 200, seeds, sel_q, sel_k)
    return dict(host=host, s=s, t=t, seeds=seeds, beta=beta, st=st, KR=KR, sel_q=sel_q, sel_k=sel_k, qsel=qsel)


def test_ba_full_size_sampled_probes(oracle_lib, ba_batch):
    b = ba_batch
    assert np.all(b["st"] == 0)
    assert np.all(b["KR"][:, 0] == 1850)
    for i, (qi, k) in enumerate(zip(b["sel_q"], b["sel_k"])):
        R = int(b["KR"][qi, 1])
        budget = oracle.budget(b["host"], int(b["s"][qi]), int(b["t"][qi]), 0.1, 200, int(b["seeds"][qi]))
        assert budget["R"] == R and budget["K"] == 1850
        want = oracle.probe_q(b["host"], int(b["s"][qi]), int(b["t"][qi]), 200, int(b["seeds"][qi]), R, [k])[0]
        assert b["qsel"][i] == want
        assert abs(b["qsel"][i] - want) <= REL_TOL * abs(want) + 1e-300


@pytest.mark.slow
def test_ba_full_size_whole_queries(oracle_lib, ba_batch):
    b = ba_batch
    for qi in (517,):
        want = oracle.query(b["host"], int(b["s"][qi]), int(b["t"][qi]), 0.1, 200, int(b["seeds"][qi]))
        assert b["beta"][qi] == want["beta"]


def test_ba_modes_agree(pw, ba):
    """Per-visit and probe-table kernels give identical estimates on BA queries."""
    host, g = ba
    s, t = uniform_pairs(host.n, 6, 77)
    seeds = query_seeds(6, 78)
    b1, st1 = pw.pw_query_batch(g.handle, s, t, 0.2, 50, seeds, pw.make_params(walk_mode=1))
    b2, st2 = pw.pw_query_batch(g.handle, s, t, 0.2, 50, seeds, pw.make_params(walk_mode=2))
    assert np.all(st1 == 0) and np.all(st2 == 0)
    np.testing.assert_array_equal(b1, b2)


def test_ba_full_size_accuracy_vs_series(ba_batch):
    """>= 95% of sampled queries within eps of beta^(L) (series oracle)."""
    b = ba_batch
    host = b["host"]
    idx = np.arange(0, 1000, 1000 // 64)[:64]
    want = exact.series_beta_many(host.row_ptr, host.col_idx, host.n, b["s"][idx], b["t"][idx], 200)
    rel = np.abs(b["beta"][idx] - want) / want
    assert (rel <= 0.1).mean() >= 0.95


def test_sharded_blocks_equal_whole_query(pw, tiny):
    """pw_query_blocks over disjoint block ranges + pw_block_median == pw_query."""
    host, g = tiny
    for s, t, seed in ((3, 77, 12345), (10, 190, 7)):
        whole = pw.pw_query(g.handle, s, t, 0.2, 32, seed)
        G = pw.pw_budget(g.handle, s, t, 0.2, 32, seed)["G"]
        parts = [pw.pw_query_blocks(g.handle, s, t, 0.2, 32, a, b, seed) for a, b in ((0, 13), (13, 30), (30, G))]
        assert pw.pw_block_median(np.concatenate(parts)) == whole


def test_stabilized_matches_oracle(pw, oracle_lib, tiny):
    """Section 4.3's doubling rule: the library's estimates and L_stop equal the oracle's."""
    host, g = tiny
    s, t = uniform_pairs(host.n, 12, 310)
    seeds = query_seeds(12, 311)
    s[3] = t[3]  # one query with s == t
    beta, L_stop, st = pw.pw_query_stabilized(g.handle, s, t, 0.2, 64, seeds)
    assert np.all(st == 0)
    for i in range(12):
        b, Ls, _ = oracle.stabilized(host, int(s[i]), int(t[i]), 0.2, 64, int(seeds[i]))
        assert beta[i] == b and L_stop[i] == Ls


def test_stabilized_ba(pw, oracle_lib, ba):
    host, g = ba
    s, t = uniform_pairs(host.n, 4, 320)
    seeds = query_seeds(4, 321)
    beta, L_stop, st = pw.pw_query_stabilized(g.handle, s, t, 0.2, 64, seeds)
    assert np.all(st == 0)
    for i in range(4):
        b, Ls, _ = oracle.stabilized(host, int(s[i]), int(t[i]), 0.2, 64, int(seeds[i]))
        assert beta[i] == b and L_stop[i] == Ls


def test_series_matches_oracle(pw, oracle_lib, tiny, ba):
    """pw_series_batch against the oracle's FP64 series (Lemma 2.3).  The GPU
    steps run in double-float (48-bit significand) and sum in a different
    order, so the bar is 1e-9 relative."""
    for host, g in (tiny, ba):
        s, t = uniform_pairs(host.n, 40, 330)
        L = np.array([0, 1, 5, 32] * 10, np.int32)
        got = pw.pw_series_batch(g.handle, s, t, L)
        for Lv in (0, 1, 5, 32):
            m = L == Lv
            want = exact.series_beta_many(host.row_ptr, host.col_idx, host.n, s[m], t[m], int(Lv))
            np.testing.assert_allclose(got[m], want, rtol=1e-9, atol=0)
    host, g = tiny
    assert pw.pw_series_batch(g.handle, [3], [3], [10])[0] == 0.0


def test_series_hub_rows_split(pw):
    """Rows of more than 1024 entries are summed in 1024-entry segments: a
    cycle of 3000 nodes with chords plus a hub of degree 2500 (three
    segments) against the oracle's series; two calls agree bit for bit."""
    n = 3000
    rng = np.random.default_rng(340)
    ring = np.arange(n)
    chords = rng.integers(0, n, size=(4000, 2))
    hub_nb = rng.choice(np.arange(1, n), size=2500, replace=False)
    u = np.concatenate([ring, chords[:, 0], np.zeros(2500, np.int64)])
    v = np.concatenate([(ring + 1) % n, chords[:, 1], hub_nb])
    host = from_edges(n, u, v, name="hub3000")
    assert int(np.diff(host.row_ptr).max()) > 2048
    g = pw.Graph(host.row_ptr, host.col_idx)
    s, t = uniform_pairs(host.n, 36, 341)
    s[:4] = 0  # queries from the hub itself
    L = np.array([0, 1, 7, 40] * 9, np.int32)
    got = pw.pw_series_batch(g.handle, s, t, L)
    assert np.array_equal(got, pw.pw_series_batch(g.handle, s, t, L))
    for Lv in (0, 1, 7, 40):
        m = L == Lv
        want = exact.series_beta_many(host.row_ptr, host.col_idx, host.n, s[m], t[m], int(Lv))
        np.testing.assert_allclose(got[m], want, rtol=1e-9, atol=0)
    g.close()
