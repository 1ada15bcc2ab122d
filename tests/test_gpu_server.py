"""Continuous-batching server (persistent kernel + device work queue): every
estimate equals the batch entry point's (hence the oracle's) bit for bit,
whether a query runs alone, in a burst, or arrives while others are on the GPU;
admission by accumulator memory; invalid queries; shutdown with work queued."""

import time

import numpy as np
import pytest

from pw_inputs import barabasi_albert, eps_uniform, grid_deleted, query_seeds, uniform_pairs

pytestmark = pytest.mark.gpu


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


def _queries(n, count, seed):
    s, t = uniform_pairs(n, count, seed)
    eps = eps_uniform(count, 0.15, 0.35, seed + 1)
    L = np.random.default_rng(seed + 2).integers(0, 40, size=count).astype(np.int32)
    seeds = query_seeds(count, seed + 3)
    return s, t, eps, L, seeds


def _serve(pw, g, s, t, eps, L, seeds, params=None, accum=1 << 26, gap_s=0.0, timeout_ms=120000):
    srv = pw.pw_server_create(g.handle, params, accum)
    try:
        tickets = []
        for i in range(s.size):
            tickets.append(pw.pw_server_submit(srv, int(s[i]), int(t[i]), float(eps[i]), int(L[i]), int(seeds[i])))
            if gap_s:
                time.sleep(gap_s)
        pw.pw_server_drain(srv, timeout_ms)
        out = np.empty(s.size)
        for i, tk in enumerate(tickets):
            st, b = pw.pw_server_poll(srv, tk)
            assert st == pw.PW_OK
            out[i] = b
        return out
    finally:
        pw.pw_server_destroy(srv)


def test_server_burst_equals_batch(pw, tiny):
    host, g = tiny
    q = _queries(host.n, 48, 500)
    want, st = pw.pw_query_batch(g.handle, *q)
    assert np.all(st == 0)
    np.testing.assert_array_equal(_serve(pw, g, *q), want)


def test_server_even_G_matches_oracle(pw, oracle_lib, tiny):
    """delta = 0.05 (G = 24, an even number of block means): the server's final
    median equals the oracle's for every query."""
    import oracle

    host, g = tiny
    s, t, eps, L, seeds = _queries(host.n, 16, 550)
    params = pw.make_params(delta=0.05)
    got = _serve(pw, g, s, t, eps, L, seeds, params=params)
    want, budgets, st = oracle.query_many(host, s, t, eps, L, seeds, oracle.budget_cfg(delta=0.05))
    assert np.all(st == 0) and np.all(budgets[s != t, 1] == 24)
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=0)
    np.testing.assert_array_equal(got, want)


def test_server_arrivals_while_busy_equal_batch(pw, tiny):
    host, g = tiny
    q = _queries(host.n, 40, 600)
    want, _ = pw.pw_query_batch(g.handle, *q)
    np.testing.assert_array_equal(_serve(pw, g, *q, gap_s=0.002), want)


def test_server_alone_equals_mix(pw, tiny):
    host, g = tiny
    s, t, eps, L, seeds = _queries(host.n, 12, 700)
    mixed = _serve(pw, g, s, t, eps, L, seeds)
    srv = pw.pw_server_create(g.handle, None, 1 << 24)
    try:
        for i in range(12):  # one query in flight at a time
            tk = pw.pw_server_submit(srv, int(s[i]), int(t[i]), float(eps[i]), int(L[i]), int(seeds[i]))
            pw.pw_server_drain(srv, 60000)
            st, b = pw.pw_server_poll(srv, tk)
            assert st == pw.PW_OK and b == mixed[i]
    finally:
        pw.pw_server_destroy(srv)


def test_server_admission_by_memory(pw, tiny):
    """A 1 MiB accumulator pool holds only a few queries at a time; the rest
    wait in the host queue and are admitted as memory frees up."""
    host, g = tiny
    q = _queries(host.n, 64, 800)
    want, _ = pw.pw_query_batch(g.handle, *q)
    np.testing.assert_array_equal(_serve(pw, g, *q, accum=1 << 20), want)


def test_server_fixed_budget(pw, tiny):
    host, g = tiny
    q = _queries(host.n, 20, 900)
    params = pw.make_params(budget_mode=pw.PW_BUDGET_FIXED, B=5, G=7, R=45)
    want, _ = pw.pw_query_batch(g.handle, *q, params)
    np.testing.assert_array_equal(_serve(pw, g, *q, params=params), want)


def test_server_invalid_and_same_node(pw, tiny):
    host, g = tiny
    srv = pw.pw_server_create(g.handle, None, 1 << 24)
    try:
        t_same = pw.pw_server_submit(srv, 3, 3, 0.2, 20, 1)
        t_bad = pw.pw_server_submit(srv, 3, 999, 0.2, 20, 1)
        t_ok = pw.pw_server_submit(srv, 3, 4, 0.2, 20, 1)
        pw.pw_server_drain(srv, 60000)
        assert pw.pw_server_poll(srv, t_same) == (pw.PW_OK, 0.0)
        with pytest.raises(pw.PWError) as e:
            pw.pw_server_poll(srv, t_bad)
        assert e.value.status == pw.PW_ERR_ARG
        st, b = pw.pw_server_poll(srv, t_ok)
        assert st == pw.PW_OK and b == pw.pw_query(g.handle, 3, 4, 0.2, 20, 1)
        with pytest.raises(pw.PWError):
            pw.pw_server_poll(srv, 10**9)  # unknown ticket
    finally:
        pw.pw_server_destroy(srv)


def test_server_collect_and_destroy_with_queue(pw, tiny):
    host, g = tiny
    s, t, eps, L, seeds = _queries(host.n, 30, 1000)
    srv = pw.pw_server_create(g.handle, None, 1 << 20)
    for i in range(30):
        pw.pw_server_submit(srv, int(s[i]), int(t[i]), float(eps[i]), int(L[i]), int(seeds[i]))
    time.sleep(0.01)
    tk, b, st, lat = pw.pw_server_collect(srv)
    assert np.all(lat >= 0)
    pw.pw_server_destroy(srv)  # queued work is cancelled, in-flight work finishes; no hang


def test_server_ticket_delivered_once(pw, tiny):
    """A result is delivered once, by poll or by collect; afterwards the ticket
    is reported as unknown instead of pending forever."""
    host, g = tiny
    s, t, eps, L, seeds = _queries(host.n, 4, 1100)
    srv = pw.pw_server_create(g.handle, None, 1 << 24)
    try:
        tks = [pw.pw_server_submit(srv, int(s[i]), int(t[i]), float(eps[i]), int(L[i]), int(seeds[i]))
               for i in range(4)]
        pw.pw_server_drain(srv, 60000)
        st, _ = pw.pw_server_poll(srv, tks[0])
        assert st == pw.PW_OK
        with pytest.raises(pw.PWError) as e1:
            pw.pw_server_poll(srv, tks[0])
        assert e1.value.status == pw.PW_ERR_ARG
        got, _, cst, _ = pw.pw_server_collect(srv)
        assert sorted(got.tolist()) == sorted(tks[1:]) and np.all(cst == 0)
        for tk in tks[1:]:
            with pytest.raises(pw.PWError) as e2:
                pw.pw_server_poll(srv, tk)
            assert e2.value.status == pw.PW_ERR_ARG
        with pytest.raises(pw.PWError):
            pw.pw_server_poll(srv, max(tks) + 100)
    finally:
        pw.pw_server_destroy(srv)


def test_server_query_larger_than_pool_fails(pw, tiny):
    """eps = 0.01 needs 185,000 probes (1.5 MB of accumulators), more than a
    1 MiB pool: the query fails with PW_ERR_NOMEM instead of waiting forever,
    and the server keeps serving."""
    host, g = tiny
    srv = pw.pw_server_create(g.handle, None, 1 << 20)
    try:
        big = pw.pw_server_submit(srv, 3, 77, 0.01, 5, 11)
        ok = pw.pw_server_submit(srv, 3, 77, 0.3, 5, 11)
        pw.pw_server_drain(srv, 60000)
        with pytest.raises(pw.PWError) as e:
            pw.pw_server_poll(srv, big)
        assert e.value.status == pw.PW_ERR_NOMEM
        assert pw.pw_server_poll(srv, ok)[0] == pw.PW_OK
    finally:
        pw.pw_server_destroy(srv)


def test_server_ba_equals_batch(pw):
    host = barabasi_albert(100_000, 5, 1)
    with pw.Graph(host.row_ptr, host.col_idx) as g:
        s, t = uniform_pairs(host.n, 16, 1100)
        seeds = query_seeds(16, 1101)
        want, st = pw.pw_query_batch(g.handle, s, t, 0.2, 100, seeds)
        assert np.all(st == 0)
        got = _serve(pw, g, s, t, np.full(16, 0.2), np.full(16, 100, np.int32), seeds, accum=1 << 28)
        np.testing.assert_array_equal(got, want)


def test_server_idle_exit_and_relaunch(pw, tiny):
    """Gaps longer than the kernel's idle window (5 ms): the grid exits between
    queries and is relaunched by the scheduler; estimates are unchanged."""
    host, g = tiny
    q = _queries(host.n, 6, 1200)
    want, _ = pw.pw_query_batch(g.handle, *q)
    np.testing.assert_array_equal(_serve(pw, g, *q, gap_s=0.02), want)


def test_server_drain_times_out_then_completes(pw):
    """A wait that runs out returns PW_ERR_TIMEOUT and leaves the server usable."""
    host = barabasi_albert(100_000, 5, 1)
    with pw.Graph(host.row_ptr, host.col_idx) as g:
        srv = pw.pw_server_create(g.handle, None, 1 << 28)
        try:
            tk = pw.pw_server_submit(srv, 10, 20000, 0.05, 200, 4242)
            with pytest.raises(pw.PWError) as e:
                pw.pw_server_drain(srv, 1)
            assert e.value.status == pw.PW_ERR_TIMEOUT
            pw.pw_server_drain(srv, 600000)
            st, b = pw.pw_server_poll(srv, tk)
            assert st == pw.PW_OK and b == pw.pw_query(g.handle, 10, 20000, 0.05, 200, 4242)
        finally:
            pw.pw_server_destroy(srv)


def test_server_tune_keeps_results(pw):
    """pw_server_tune times every walk-kernel policy on a sample and keeps the
    fastest; estimates after tuning equal the batch entry point's, and the
    policies it timed all produced the batch's estimates too (it polls them)."""
    h = barabasi_albert(20_000, 5, 21)
    with pw.Graph(h.row_ptr, h.col_idx) as g:
        s, t = uniform_pairs(h.n, 12, 960)
        seeds = query_seeds(12, 961)
        want, st = pw.pw_query_batch(g.handle, s, t, 0.2, 40, seeds)
        assert np.all(st == 0)
        pw.pw_autotune(g.handle, s[:4], t[:4], 0.2, 40, seeds[:4])
        srv = pw.pw_server_create(g.handle, None, 1 << 26)
        try:
            r = pw.pw_server_tune(srv, s[:6], t[:6], 0.2, 40, seeds[:6])
            assert r["policy"] in (0, 1, 2, 3) and r["occupancy"] == 4
            assert all(r["queries_per_s"][p] > 0 for p in (0, 1, 2, 3))
            assert r["occupancy_qps"] == [0.0, 0.0]
            assert r["queries_per_s"][r["policy"]] == max(r["queries_per_s"])
            tk = [pw.pw_server_submit(srv, int(s[i]), int(t[i]), 0.2, 40, int(seeds[i])) for i in range(12)]
            pw.pw_server_drain(srv, 60000)
            got = [pw.pw_server_poll(srv, x)[1] for x in tk]
        finally:
            pw.pw_server_destroy(srv)
        np.testing.assert_array_equal(got, want)


def test_server_tune_occupancy_without_table(pw):
    """On a graph whose probe table does not fit in shared memory (n above
    1,638,336) every policy runs the same per-visit jobs, so pw_server_tune times
    the server kernel at 2 and at 3 blocks/SM and keeps the faster.  The tuner
    requires both variants to give the same estimates bit for bit, and the
    server's estimates after tuning equal the batch entry point's."""
    h = grid_deleted(1400, 0.05, 7)
    assert h.n > 1_638_336
    with pw.Graph(h.row_ptr, h.col_idx) as g:
        s, t = uniform_pairs(h.n, 8, 970)
        seeds = query_seeds(8, 971)
        want, st = pw.pw_query_batch(g.handle, s, t, 0.2, 60, seeds)
        assert np.all(st == 0)
        srv = pw.pw_server_create(g.handle, None, 1 << 26)
        try:
            r = pw.pw_server_tune(srv, s[:4], t[:4], 0.2, 60, seeds[:4])
            assert r["policy"] == 0 and r["occupancy"] in (2, 3)
            assert all(q > 0 for q in r["occupancy_qps"])
            assert r["queries_per_s"][0] == max(r["occupancy_qps"])
            assert r["queries_per_s"][1:] == [0.0, 0.0, 0.0]
            tk = [pw.pw_server_submit(srv, int(s[i]), int(t[i]), 0.2, 60, int(seeds[i])) for i in range(8)]
            pw.pw_server_drain(srv, 120000)
            got = [pw.pw_server_poll(srv, x)[1] for x in tk]
        finally:
            pw.pw_server_destroy(srv)
        np.testing.assert_array_equal(got, want)

