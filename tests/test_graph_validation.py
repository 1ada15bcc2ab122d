"""pw_graph_load's checks of Section 2.1's assumptions (undirected, simple,
connected, no isolated node) run on the host before any CUDA call, so they are
tested here without a GPU: every malformed CSR is rejected with PW_ERR_GRAPH
(or PW_ERR_ARG) and a message naming the fault.  A well-formed graph on a
machine without a usable GPU fails with PW_ERR_CUDA: there is no CPU path."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def pw():
    from paper_2512_05460_gb300 import build

    build.build()
    from paper_2512_05460_gb300 import probewalk

    probewalk.lib()
    return probewalk


def _csr(n, edges):
    """Symmetric CSR with sorted rows from undirected edges."""
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(a) for a in adj])
    col = np.array([u for a in adj for u in sorted(a)], np.int32)
    return rp, col


TRIANGLE_TAIL = [(0, 1), (1, 2), (0, 2), (2, 3)]


def _rejects(pw, rp, col, status, words, loader="pw_graph_load"):
    with pytest.raises(pw.PWError) as e:
        getattr(pw, loader)(rp, col, 0, 0)
    assert e.value.status == status
    for w in words:
        assert w in str(e.value), (w, str(e.value))


def test_malformed_csr_is_rejected(pw):
    rp, col = _csr(4, TRIANGLE_TAIL)
    bad = rp.copy()
    bad[0] = 1
    _rejects(pw, bad, col, pw.PW_ERR_GRAPH, ["row_ptr must start at 0"])
    bad = rp.copy()
    bad[2], bad[3] = bad[3], bad[2]
    _rejects(pw, bad, col, pw.PW_ERR_GRAPH, ["not monotone"])
    c = col.copy()
    c[0] = 9
    _rejects(pw, rp, c, pw.PW_ERR_GRAPH, ["out of range"])
    c = col.copy()
    c[0] = 0  # node 0's first neighbour becomes itself
    _rejects(pw, rp, c, pw.PW_ERR_GRAPH, ["self-loop at node 0"])
    c = col.copy()
    c[0], c[1] = c[1], c[0]  # row 0 out of order
    _rejects(pw, rp, c, pw.PW_ERR_GRAPH, ["row 0 is not strictly increasing"])
    rp5, col5 = _csr(5, TRIANGLE_TAIL)  # node 4 has no edge
    _rejects(pw, rp5, col5, pw.PW_ERR_GRAPH, ["isolated node 4"])
    rp6, col6 = _csr(6, TRIANGLE_TAIL + [(4, 5)])
    _rejects(pw, rp6, col6, pw.PW_ERR_GRAPH, ["not connected"])


def test_directed_and_duplicate_edges_are_rejected(pw):
    # 0 -> 1 without 1 -> 0
    rp = np.array([0, 2, 3, 5, 6], np.int64)
    col = np.array([1, 2, 2, 0, 1, 2], np.int32)  # rows: 0:{1,2} 1:{2} 2:{0,1} 3:{2}
    _rejects(pw, rp, col, pw.PW_ERR_GRAPH, ["has no reverse"])
    # a duplicate entry in a row is a multi-edge
    rp, col = _csr(4, TRIANGLE_TAIL)
    rp2 = rp.copy()
    rp2[1:] += 1
    col2 = np.insert(col, 1, col[0])
    _rejects(pw, rp2, col2, pw.PW_ERR_GRAPH, ["row 0 is not strictly increasing"])


def test_bad_sizes_are_rejected(pw):
    _rejects(pw, np.array([0, 0], np.int64), np.zeros(0, np.int32), pw.PW_ERR_ARG, ["n must lie in"])
    _rejects(pw, np.array([0, 0, 0], np.int64), np.zeros(0, np.int32), pw.PW_ERR_ARG, ["nnz must lie in"])


def test_32_bit_loader_checks_the_same(pw):
    rp5, col5 = _csr(5, TRIANGLE_TAIL)
    _rejects(pw, rp5.astype(np.int32), col5, pw.PW_ERR_GRAPH, ["isolated node 4"], loader="pw_graph_load32")


def test_valid_graph_needs_a_gpu(pw):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the load would succeed")
    rp, col = _csr(4, TRIANGLE_TAIL)
    with pytest.raises(pw.PWError) as e:
        pw.pw_graph_load(rp, col, 0, 0)
    assert e.value.status == pw.PW_ERR_CUDA
