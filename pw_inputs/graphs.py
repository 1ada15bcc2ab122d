"""Seeded undirected simple graphs in sorted CSR form.

Every generator returns a :class:`CSRGraph` whose rows are strictly increasing,
symmetric, free of self-loops and duplicates, and (unless stated) restricted
to the largest connected component with nodes relabelled in increasing order
of their original ids.  The families mirror the synthetic stand-ins for the
paper's SNAP/SOMAR networks (Section 4.1, Table 2; heavy-tailed degrees,
Appendix A.1): Erdos-Renyi unioned with a cycle, Barabasi-Albert preferential
attachment, R-MAT/Kronecker, and a 2-D grid with random edge deletions.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class CSRGraph:
    n: int
    row_ptr: np.ndarray  # int64, length n+1
    col_idx: np.ndarray  # int32, length nnz
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    @property
    def d_min(self) -> int:
        return int(self.degrees.min())

    @property
    def d_max(self) -> int:
        return int(self.degrees.max())

    def row_ptr32(self) -> np.ndarray:
        if self.nnz >= 2**31:
            raise ValueError("nnz does not fit int32 offsets")
        return self.row_ptr.astype(np.int32)

    def is_bipartite(self) -> bool:
        """Two-colour the graph by breadth-first search."""
        from scipy.sparse import csr_matrix
        from scipy.sparse.csgraph import breadth_first_order

        a = csr_matrix(
            (np.ones(self.nnz, np.int8), self.col_idx, self.row_ptr), shape=(self.n, self.n)
        )
        colour = np.full(self.n, -1, np.int8)
        for root in range(self.n):
            if colour[root] >= 0:
                continue
            order, pred = breadth_first_order(a, root, directed=False, return_predecessors=True)
            colour[root] = 0
            for v in order[1:]:
                colour[v] = 1 - colour[pred[v]]
        src = np.repeat(np.arange(self.n), self.degrees)
        return bool(np.all(colour[src] != colour[self.col_idx]))


def _csr_from_directed(n: int, src: np.ndarray, dst: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    order = np.lexsort((dst, src))
    src = src[order]
    dst = dst[order]
    counts = np.bincount(src, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, dst.astype(np.int32)


def from_edges(n: int, u, v, name: str = "", keep_lcc: bool = True, meta=None) -> CSRGraph:
    """Symmetrise, drop self-loops and duplicates, optionally keep the largest component."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    key = np.unique(a * n + b)
    a = key // n
    b = key % n
    del key
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    del a, b
    row_ptr, col_idx = _csr_from_directed(n, src, dst)
    del src, dst
    g = CSRGraph(n, row_ptr, col_idx, name, dict(meta or {}))
    if keep_lcc:
        g = largest_component(g)
    return g


def largest_component(g: CSRGraph) -> CSRGraph:
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components

    a = csr_matrix((np.ones(g.nnz, np.int8), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    ncomp, label = connected_components(a, directed=False)
    deg = g.degrees
    if ncomp == 1 and deg.min() > 0:
        return g
    sizes = np.bincount(label)
    big = int(np.argmax(sizes))
    keep = label == big
    new_id = np.full(g.n, -1, np.int64)
    new_id[keep] = np.arange(int(keep.sum()))
    src = np.repeat(np.arange(g.n), deg)
    m = keep[src]
    src_new = new_id[src[m]]
    dst_new = new_id[g.col_idx[m]]
    n2 = int(keep.sum())
    row_ptr, col_idx = _csr_from_directed(n2, src_new, dst_new)
    meta = dict(g.meta)
    meta["lcc_of"] = g.n
    return CSRGraph(n2, row_ptr, col_idx, g.name, meta)


def complete_graph(n: int) -> CSRGraph:
    i, j = np.triu_indices(n, 1)
    return from_edges(n, i, j, name=f"K{n}", keep_lcc=False)


def cycle_graph(n: int) -> CSRGraph:
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, name=f"C{n}", keep_lcc=False)


def path_graph(n: int) -> CSRGraph:
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, name=f"P{n}", keep_lcc=False)


def er_cycle(n: int = 200, p: float = 8 / 199, seed: int = 0) -> CSRGraph:
    """G(n, p) unioned with the cycle 0-1-...-(n-1)-0 (which keeps it connected)."""
    rng = np.random.default_rng(seed)
    i, j = np.triu_indices(n, 1)
    pick = rng.random(i.size) < p
    ring = np.arange(n)
    u = np.concatenate([i[pick], ring])
    v = np.concatenate([j[pick], (ring + 1) % n])
    return from_edges(n, u, v, name=f"er{n}-cycle", meta={"p": p, "seed": seed})


def barabasi_albert(n: int = 100_000, m: int = 5, seed: int = 1) -> CSRGraph:
    """Preferential attachment: start from a clique on m+1 nodes, then every new
    node links to m distinct existing nodes drawn with probability proportional
    to their current degree."""
    rng = np.random.default_rng(seed)
    m0 = m + 1
    n_edges = m0 * (m0 - 1) // 2 + (n - m0) * m
    src = np.empty(n_edges, np.int64)
    dst = np.empty(n_edges, np.int64)
    pool = np.empty(2 * n_edges, np.int64)
    e = 0
    for i in range(m0):
        for j in range(i + 1, m0):
            src[e], dst[e] = i, j
            pool[2 * e], pool[2 * e + 1] = i, j
            e += 1
    for v in range(m0, n):
        filled = 2 * e
        chosen: list[int] = []
        while len(chosen) < m:
            for c in pool[rng.integers(0, filled, size=2 * m)].tolist():
                if c not in chosen:
                    chosen.append(c)
                    if len(chosen) == m:
                        break
        for c in chosen:
            src[e], dst[e] = v, c
            pool[2 * e], pool[2 * e + 1] = v, c
            e += 1
    return from_edges(n, src, dst, name=f"ba{n}-m{m}", meta={"m": m, "seed": seed})


def rmat(scale: int = 20, edge_factor: int = 16, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 2,
         chunk: int = 1 << 22) -> CSRGraph:
    """R-MAT/Kronecker edges on 2**scale nodes; symmetrised, deduplicated,
    self-loops dropped, largest component kept."""
    a, b, c, _ = abcd
    n = 1 << scale
    n_edges = edge_factor * n
    rng = np.random.default_rng(seed)
    us, vs = [], []
    for start in range(0, n_edges, chunk):
        size = min(chunk, n_edges - start)
        u = np.zeros(size, np.int64)
        v = np.zeros(size, np.int64)
        for level in range(scale):
            r = rng.random(size)
            bit = np.int64(1) << np.int64(scale - 1 - level)
            u_hi = r >= a + b
            v_hi = ((r >= a) & (r < a + b)) | (r >= a + b + c)
            u |= np.where(u_hi, bit, 0)
            v |= np.where(v_hi, bit, 0)
        us.append(u)
        vs.append(v)
    u = np.concatenate(us)
    del us
    v = np.concatenate(vs)
    del vs
    return from_edges(n, u, v, name=f"rmat{scale}-ef{edge_factor}",
                      meta={"scale": scale, "edge_factor": edge_factor, "abcd": tuple(abcd), "seed": seed})


def grid_deleted(side: int = 2000, frac: float = 0.05, seed: int = 3) -> CSRGraph:
    """side x side grid (4-neighbour) with round(frac * edges) edges deleted
    uniformly at random; largest component kept.  The result is bipartite."""
    rng = np.random.default_rng(seed)
    idx = np.arange(side * side, dtype=np.int64).reshape(side, side)
    hu, hv = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    vu, vv = idx[:-1, :].ravel(), idx[1:, :].ravel()
    u = np.concatenate([hu, vu])
    v = np.concatenate([hv, vv])
    n_del = int(round(frac * u.size))
    drop = rng.choice(u.size, size=n_del, replace=False)
    keep = np.ones(u.size, bool)
    keep[drop] = False
    return from_edges(side * side, u[keep], v[keep], name=f"grid{side}-del{frac}",
                      meta={"side": side, "frac": frac, "seed": seed})


_NATIVE = None


def _native_lib():
    """Build (once) and load the C R-MAT generator (rmat_gen.c, gcc + OpenMP)."""
    global _NATIVE
    if _NATIVE is None:
        import ctypes
        import os
        import subprocess

        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "rmat_gen.c")
        out_dir = os.path.join(here, "_lib")
        so = os.path.join(out_dir, "libpwgen.so")
        os.makedirs(out_dir, exist_ok=True)
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            tmp = so + f".tmp{os.getpid()}"
            subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src], check=True)
            os.replace(tmp, so)
        lib = ctypes.CDLL(so)
        P = ctypes.POINTER
        lib.pwgen_rmat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_uint64, ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_int64),
                                   P(P(ctypes.c_int64)), P(P(ctypes.c_int32))]
        lib.pwgen_rmat.restype = ctypes.c_int
        lib.pwgen_free.argtypes = [ctypes.c_void_p]
        lib.pwgen_free.restype = None
        _NATIVE = lib
    return _NATIVE


def rmat_native(scale: int = 24, edge_factor: int = 16, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 4,
                threads: int = 0) -> CSRGraph:
    """R-MAT at large scales with the C generator (counter-based draws, so the
    graph does not depend on the thread count): symmetrised, deduplicated,
    self-loops dropped, largest component kept and relabelled."""
    import ctypes

    lib = _native_lib()
    a, b, c, _ = abcd
    n, m = ctypes.c_int64(), ctypes.c_int64()
    rp = ctypes.POINTER(ctypes.c_int64)()
    ci = ctypes.POINTER(ctypes.c_int32)()
    if lib.pwgen_rmat(scale, edge_factor, a, b, c, seed, threads, ctypes.byref(n), ctypes.byref(m),
                      ctypes.byref(rp), ctypes.byref(ci)) != 0:
        raise MemoryError("R-MAT generation failed")
    try:
        row_ptr = np.ctypeslib.as_array(rp, shape=(n.value + 1,)).copy()
        col_idx = np.ctypeslib.as_array(ci, shape=(max(m.value, 1),))[: m.value].copy()
    finally:
        lib.pwgen_free(ctypes.cast(rp, ctypes.c_void_p))
        lib.pwgen_free(ctypes.cast(ci, ctypes.c_void_p))
    return CSRGraph(n.value, row_ptr, col_idx, f"rmat{scale}-ef{edge_factor}-native",
                    {"scale": scale, "edge_factor": edge_factor, "abcd": tuple(abcd), "seed": seed, "lcc_of": 1 << scale})


WORKLOADS = {
    "tiny-er200": lambda: er_cycle(200, 8 / 199, 0),
    "ba-1e5": lambda: barabasi_albert(100_000, 5, 1),
    "rmat-20": lambda: rmat(20, 16, (0.57, 0.19, 0.19, 0.05), 2),
    "grid-2000": lambda: grid_deleted(2000, 0.05, 3),
    "rmat-24": lambda: rmat_native(24, 16, (0.57, 0.19, 0.19, 0.05), 4),
}


def workload_graph(name: str) -> CSRGraph:
    return WORKLOADS[name]()
