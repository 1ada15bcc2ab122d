"""pw_query_batch_noalloc: the batch entry point for callers that must not
allocate device memory while they serve queries.  It takes its scratch from a
static device array instead of cudaMalloc; its estimates must equal those of
pw_query_batch (the allocating entry point) on two calls in a row, because
the array is shared and reused from call to call.  This file is collected
last so that a failure here cannot stop the rest of a -x run."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    from paper_2512_05460_gb300 import build

    build.build()
    from paper_2512_05460_gb300 import probewalk as pw
    from pw_inputs import er_cycle, eps_uniform, query_seeds, uniform_pairs

    host = er_cycle(200, 8 / 199, 0)
    g = pw.Graph(host.row_ptr, host.col_idx, device=0)
    n = 24
    s, t = uniform_pairs(host.n, n, 31)
    eps = eps_uniform(n, 0.15, 0.3, 32)
    L = np.random.default_rng(33).integers(0, 40, size=n).astype(np.int32)
    seeds = query_seeds(n, 34)
    yield torch, pw, host, g, (s, t, eps, L, seeds)
    g.close()


@pytest.mark.parametrize("walk_mode", [1, 2])
def test_noalloc_matches_allocating_entry_point_twice(setup, walk_mode):
    """Both walk kernels (per-visit probe evaluation, per-probe table), each
    with its own offsets into the shared array."""
    torch, pw, host, g, (s, t, eps, L, seeds) = setup
    params = pw.make_params(walk_mode=walk_mode)
    want, wst = pw.pw_query_batch(g.handle, s, t, eps, L, seeds, params)
    assert np.all(wst == 0)
    dev = torch.device("cuda:0")
    n = s.size
    d = [torch.from_numpy(a).to(dev) for a in (s, t, eps, L, seeds.view(np.int64))]
    stream = torch.cuda.Stream()
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        beta = torch.full((n,), -1.0, dtype=torch.float64, device=dev)
        status = torch.full((n,), 99, dtype=torch.int32, device=dev)
        pw.pw_query_batch_noalloc(g.handle, n, *d, beta, status, params, stream=stream)
        stream.synchronize()
        assert pw.pw_profile(g.handle, enable=False, reset=False)["walk_mode"] == walk_mode
        got = beta.cpu().numpy()
        assert int(status.abs().sum()) == 0
        np.testing.assert_allclose(got, want, rtol=REL_TOL, atol=0)


def test_noalloc_rejects_batches_beyond_the_static_scratch(setup):
    torch, pw, host, g, _ = setup
    dev = torch.device("cuda:0")
    n = 4
    s = torch.zeros(n, dtype=torch.int64, device=dev)
    t = torch.ones(n, dtype=torch.int64, device=dev)
    eps = torch.full((n,), 0.01, dtype=torch.float64, device=dev)  # B = 10,000 probes per query
    L = torch.full((n,), 32, dtype=torch.int32, device=dev)
    beta = torch.empty(n, dtype=torch.float64, device=dev)
    status = torch.empty(n, dtype=torch.int32, device=dev)
    with pytest.raises(pw.PWError) as err:
        pw.pw_query_batch_noalloc(g.handle, n, s, t, eps, L, None, beta, status)
    assert err.value.status == pw.PW_ERR_NOMEM
