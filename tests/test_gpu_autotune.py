"""Walk-kernel autotuner (pw_autotune) on the GPU.

The two walk kernels (per-visit probe evaluation, per-probe shared-memory
table) compute the same U_p bit for bit, so tuning may change only which kernel
runs: the tests check that the fitted model is sane, that the auto mode then
runs the kernel the model picks, and that every mode gives identical estimates.
"""
import numpy as np
import pytest

from pw_inputs import barabasi_albert, grid_deleted, query_seeds, uniform_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_2512_05460_gb300 import build

    build.build()
    from paper_2512_05460_gb300 import probewalk

    probewalk.lib()
    return probewalk


def _batch(pw, g, s, t, eps, L, seeds, mode):
    beta, st = pw.pw_query_batch(g.handle, s, t, eps, L, seeds, pw.make_params(walk_mode=mode))
    assert np.all(st == 0)
    prof = pw.pw_profile(g.handle, enable=False, reset=True)
    return beta, prof["walk_mode"]


def test_autotune_fits_and_auto_mode_follows_it(pw):
    h = barabasi_albert(20_000, 5, 11)
    g = pw.Graph(h.row_ptr, h.col_idx)
    s, t = uniform_pairs(h.n, 6, 901)
    seeds = query_seeds(6, 902)
    eps, L = 0.15, 60
    r = pw.pw_autotune(g.handle, s, t, eps, L, seeds)
    assert r["table_available"] == 1
    assert r["visit_ns"] > 0 and all(x > 0 for x in r["sample_ms"])
    assert r["table_probe_ns"] >= 0 and r["table_visit_ns"] >= 0
    assert r["table_probe_ns"] + r["table_visit_ns"] > 0
    assert r["sample_mode"] in (1, 2)
    assert r["visit_occupancy"] in (1, 3) and r["table_threads"] in (256, 512, 1024)
    # the auto mode gives each query the kernel the fitted model picks for it
    _, _, KR, _ = pw.pw_debug_batch_probe_q(g.handle, s, t, eps, L, seeds, [], [])
    gain = r["visit_ns"] - r["table_visit_ns"]
    table = [r["table_probe_ns"] < 2.0 * float(R) * (L + 1) * gain for K, R in KR if K > 0]
    want_mode = (1 if not all(table) else 0) | (2 if any(table) else 0)
    # ... unless the timed policy check kept "all per-visit" or "all table"
    assert r["policy"] in (0, 1, 2) and all(x > 0 for x in r["policy_ms"])
    # the fastest, except that a single-kernel policy within 1 % of the model is preferred to it
    if r["policy"] == 0:
        assert r["policy_ms"][0] == min(r["policy_ms"]) and min(r["policy_ms"][1:]) > 1.01 * r["policy_ms"][0]
    else:
        assert r["policy_ms"][r["policy"]] <= 1.01 * min(r["policy_ms"])
    if r["policy"] != 0:
        want_mode = r["policy"]
    # L2 window: none and the gathered records timed (fused layout: no node-record window)
    timed = [x for x in r["window_ms"] if x > 0]
    assert r["window_ms"][0] > 0 and r["window_ms"][2] == 0
    assert r["l2_window"] in (0, 1)
    if r["l2_window"]:
        assert r["window_ms"][r["l2_window"]] == min(timed) < 0.98 * r["window_ms"][0]
    pw.pw_profile(g.handle, enable=True, reset=True)
    b0, m0 = _batch(pw, g, s, t, eps, L, seeds, 0)
    assert m0 == want_mode
    b1, m1 = _batch(pw, g, s, t, eps, L, seeds, 1)
    b2, m2 = _batch(pw, g, s, t, eps, L, seeds, 2)
    assert (m1, m2) == (1, 2)
    assert np.array_equal(b0, b1) and np.array_equal(b1, b2)
    # estimates do not depend on whether the graph was tuned
    g2 = pw.Graph(h.row_ptr, h.col_idx)
    b_untuned, _ = pw.pw_query_batch(g2.handle, s, t, eps, L, seeds)
    assert np.array_equal(b_untuned, b0)
    g2.close()
    g.close()


def test_autotune_without_table(pw):
    """n > 1,638,336: the 1-bit table (n/8 bytes) exceeds its 200 KB of shared
    memory, so only the per-visit kernel is timed and the auto mode stays
    per-visit."""
    h = grid_deleted(1300, 0.05, 12)
    assert h.n > 1_638_336
    g = pw.Graph(h.row_ptr, h.col_idx)
    s, t = uniform_pairs(h.n, 4, 903)
    seeds = query_seeds(4, 904)
    r = pw.pw_autotune(g.handle, s, t, 0.2, 20, seeds)
    assert r["table_available"] == 0 and r["sample_mode"] == 1
    assert r["visit_ns"] > 0 and r["table_probe_ns"] == 0 and r["table_visit_ns"] == 0
    timed = [x for x in r["window_ms"] if x > 0]
    assert r["window_ms"][0] > 0 and r["l2_window"] in (0, 1, 2)
    if r["l2_window"]:
        assert r["window_ms"][r["l2_window"]] == min(timed) < 0.98 * r["window_ms"][0]
    pw.pw_profile(g.handle, enable=True, reset=True)
    b0, m0 = _batch(pw, g, s, t, 0.2, 20, seeds, 0)
    assert m0 == 1
    b1, _ = _batch(pw, g, s, t, 0.2, 20, seeds, 1)
    assert np.array_equal(b0, b1)
    g.close()


def test_autotune_rejects_bad_sample(pw):
    h = barabasi_albert(2_000, 3, 13)
    g = pw.Graph(h.row_ptr, h.col_idx)
    with pytest.raises(pw.PWError):
        pw.pw_autotune(g.handle, np.zeros(0, np.int64), np.zeros(0, np.int64), 0.1, 10)
    with pytest.raises(pw.PWError):
        pw.pw_autotune(g.handle, [0], [h.n + 5], 0.1, 10)
    g.close()


@pytest.mark.parametrize("layout", ["fused", "split"])
def test_l2_window_keeps_estimates(pw, layout):
    """An L2 access-policy window changes only what stays in L2: with each
    window the batch (eager, captured, replayed) and the server give the
    estimates of the launches without one; on the fused layout the
    node-record window is rejected."""
    h = barabasi_albert(20_000, 5, 31)
    flags = pw.LOAD_FUSED if layout == "fused" else pw.LOAD_SPLIT
    g = pw.Graph(h.row_ptr, h.col_idx, flags=flags)
    s, t = uniform_pairs(h.n, 6, 990)
    seeds = query_seeds(6, 991)
    want, st = pw.pw_query_batch(g.handle, s, t, 0.2, 40, seeds)
    assert np.all(st == 0)
    windows = (1,) if layout == "fused" else (1, 2)
    if layout == "fused":
        with pytest.raises(pw.PWError):
            pw.pw_graph_set_l2_window(g.handle, 2)
    with pytest.raises(pw.PWError):
        pw.pw_graph_set_l2_window(g.handle, 3)
    for w in windows:
        pw.pw_graph_set_l2_window(g.handle, w)
        for _ in range(3):  # eager, then captured into a CUDA graph, then replayed
            got, st = pw.pw_query_batch(g.handle, s, t, 0.2, 40, seeds)
            assert np.all(st == 0)
            np.testing.assert_array_equal(got, want)
        srv = pw.pw_server_create(g.handle, None, 1 << 26)
        try:
            tk = [pw.pw_server_submit(srv, int(s[i]), int(t[i]), 0.2, 40, int(seeds[i])) for i in range(6)]
            pw.pw_server_drain(srv, 60000)
            got = [pw.pw_server_poll(srv, x)[1] for x in tk]
        finally:
            pw.pw_server_destroy(srv)
        np.testing.assert_array_equal(got, want)
    pw.pw_graph_set_l2_window(g.handle, 0)
    got, _ = pw.pw_query_batch(g.handle, s, t, 0.2, 40, seeds)
    np.testing.assert_array_equal(got, want)
    g.close()

