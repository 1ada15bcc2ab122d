"""Thin ctypes binding of libprobewalk.so (see include/probewalk.h).

Every function here has the name of the C entry point it wraps and only
marshals arguments: numpy arrays for host memory, torch CUDA tensors (or raw
device addresses) for device memory, a CUDA stream handle for the device
call.  All computation happens in the library's CUDA kernels.  There is no
fallback: if the library was not built, loading fails with an error.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libprobewalk.so")

PW_OK, PW_PENDING = 0, 1
PW_ERR_ARG, PW_ERR_GRAPH, PW_ERR_NOMEM, PW_ERR_CUDA = -1, -2, -3, -4
PW_ERR_TIMEOUT, PW_ERR_CANCELLED, PW_ERR_FULL, PW_ERR_INTERNAL = -5, -6, -7, -8
PW_BUDGET_PILOT, PW_BUDGET_THEORY, PW_BUDGET_SCALED, PW_BUDGET_FIXED, PW_BUDGET_ADAPTIVE = 0, 1, 2, 3, 4
TAG_WALK, TAG_WALK_PILOT, TAG_PROBE, TAG_PROBE_PILOT = 1, 2, 3, 4
# pw_graph_load flags: skip the connectivity check; force the fused or the split walk layout
LOAD_NO_CONNECTIVITY, LOAD_FUSED, LOAD_SPLIT = 1, 2, 4

_STATUS_NAMES = {0: "PW_OK", 1: "PW_PENDING", -1: "PW_ERR_ARG", -2: "PW_ERR_GRAPH", -3: "PW_ERR_NOMEM",
                 -4: "PW_ERR_CUDA", -5: "PW_ERR_TIMEOUT", -6: "PW_ERR_CANCELLED", -7: "PW_ERR_FULL",
                 -8: "PW_ERR_INTERNAL"}


class PWError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class pw_params(ctypes.Structure):
    _fields_ = [
        ("delta", ctypes.c_double),
        ("budget_mode", ctypes.c_int32),
        ("pilot_K0", ctypes.c_int32),
        ("pilot_R0", ctypes.c_int32),
        ("reserved0", ctypes.c_int32),
        ("c_B", ctypes.c_double),
        ("c_R", ctypes.c_double),
        ("B", ctypes.c_uint64),
        ("G", ctypes.c_uint64),
        ("R", ctypes.c_uint64),
        ("R_max", ctypes.c_uint64),
        ("seed", ctypes.c_uint64),
        ("walk_mode", ctypes.c_int32),
        ("reserved1", ctypes.c_int32),
        ("z", ctypes.c_double),
        ("cap", ctypes.c_double),
    ]


def make_params(**kw) -> pw_params:
    p = pw_params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class pw_server_tune_result(ctypes.Structure):
    _fields_ = [("queries_per_s", ctypes.c_double * 4), ("occupancy_qps", ctypes.c_double * 2),
                ("policy", ctypes.c_int32), ("occupancy", ctypes.c_int32)]


class pw_profile_stats(ctypes.Structure):
    _fields_ = [
        ("walk_ms", ctypes.c_double),
        ("pilot_ms", ctypes.c_double),
        ("finish_ms", ctypes.c_double),
        ("walk_launches", ctypes.c_uint64),
        ("transitions", ctypes.c_uint64),
        ("pilot_transitions", ctypes.c_uint64),
        ("queries", ctypes.c_uint64),
        ("walk_mode", ctypes.c_int32),
        ("layout", ctypes.c_int32),
        ("series_ms", ctypes.c_double),
        ("series_steps", ctypes.c_uint64),
    ]


class pw_tune_result(ctypes.Structure):
    _fields_ = [
        ("visit_ns", ctypes.c_double),
        ("table_visit_ns", ctypes.c_double),
        ("table_probe_ns", ctypes.c_double),
        ("sample_ms", ctypes.c_double * 3),
        ("table_available", ctypes.c_int32),
        ("sample_mode", ctypes.c_int32),
        ("visit_occupancy", ctypes.c_int32),
        ("table_threads", ctypes.c_int32),
        ("policy_ms", ctypes.c_double * 3),
        ("policy", ctypes.c_int32),
        ("l2_window", ctypes.c_int32),
        ("window_ms", ctypes.c_double * 3),
    ]


_lib = None
_lock = threading.Lock()

P = ctypes.POINTER
_vp = ctypes.c_void_p
_i64, _i32, _u64, _u32, _dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double

# name -> (restype, argtypes)
SIGNATURES = {
    "pw_graph_load": (_i32, [_i64, P(_i64), P(_i32), _i64, _i32, _u32, P(_vp)]),
    "pw_graph_load32": (_i32, [_i32, P(_i32), P(_i32), _i32, _i32, _u32, P(_vp)]),
    "pw_graph_free": (None, [_vp]),
    "pw_graph_set_l2_window": (_i32, [_vp, _i32]),
    "pw_graph_info": (_i32, [_vp, P(_i64), P(_i64), P(_i32), P(_i32), P(_i32)]),
    "pw_budget": (_i32, [_vp, _i64, _i64, _dbl, _i32, P(_u64), P(pw_params), P(_u64), P(_u64), P(_u64), P(_u64)]),
    "pw_default_seed": (_u64, [_u64, _i64, _i64, _dbl, _i32]),
    "pw_query": (_i32, [_vp, _i64, _i64, _dbl, _i32, P(_u64), P(pw_params), P(_dbl)]),
    "pw_query_batch": (_i32, [_vp, _i64, P(_i64), P(_i64), P(_dbl), P(_i32), P(_u64), P(pw_params), P(_dbl),
                              P(_i32)]),
    "pw_query_batch_device": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, P(pw_params), _vp, _vp, _vp]),
    "pw_query_batch_noalloc": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, P(pw_params), _vp, _vp, _vp]),
    "pw_query_stabilized": (_i32, [_vp, _i64, P(_i64), P(_i64), P(_dbl), _i32, P(_u64), P(pw_params), P(_dbl),
                                   P(_i32), P(_i32)]),
    "pw_level_seed": (_u64, [_u64, _i32]),
    "pw_series_batch": (_i32, [_vp, _i64, P(_i64), P(_i64), P(_i32), P(_dbl)]),
    "pw_query_blocks": (_i32, [_vp, _i64, _i64, _dbl, _i32, P(_u64), P(pw_params), _i64, _i64, P(_dbl)]),
    "pw_block_median": (_i32, [P(_dbl), _i64, P(_dbl)]),
    "pw_server_create": (_i32, [_vp, P(pw_params), ctypes.c_size_t, P(_vp)]),
    "pw_server_submit": (_i32, [_vp, _i64, _i64, _dbl, _i32, P(_u64), P(_u64)]),
    "pw_server_poll": (_i32, [_vp, _u64, P(_dbl)]),
    "pw_server_collect": (_i32, [_vp, _i64, P(_u64), P(_dbl), P(_i32), P(_dbl), P(_i64)]),
    "pw_server_drain": (_i32, [_vp, _i64]),
    "pw_server_tune": (_i32, [_vp, _i64, P(_i64), P(_i64), P(_dbl), P(_i32), P(_u64), P(pw_server_tune_result)]),
    "pw_server_destroy": (_i32, [_vp]),
    "pw_debug_philox": (_i32, [_vp, P(_u32), P(_u32), P(_u32)]),
    "pw_debug_probe": (_i32, [_vp, _u64, _u32, _u32, P(ctypes.c_int8), P(_i32)]),
    "pw_debug_walk": (_i32, [_vp, _i64, _i32, _u64, _u64, _u32, P(_i64)]),
    "pw_debug_gather_peak": (_i32, [_vp, _i32, P(_dbl)]),
    "pw_debug_exact_sum": (_i32, [_vp, P(ctypes.c_float), _i64, P(_dbl), P(_dbl)]),
    "pw_debug_query": (_i32, [_vp, _i64, _i64, _dbl, _i32, P(_u64), P(pw_params), P(_dbl), P(_u64), P(_dbl),
                              P(_dbl), _i64, P(ctypes.c_float), _i64, P(_u32)]),
    "pw_debug_batch_probe_q": (_i32, [_vp, _i64, P(_i64), P(_i64), P(_dbl), P(_i32), P(_u64), P(pw_params), P(_dbl),
                                      P(_i32), P(_u64), _i64, P(_i64), P(_i64), P(_dbl)]),
    "pw_profile": (_i32, [_vp, _i32, _i32, P(pw_profile_stats)]),
    "pw_autotune": (_i32, [_vp, _i64, P(_i64), P(_i64), P(_dbl), P(_i32), P(_u64), P(pw_params), P(pw_tune_result)]),
    "pw_launch_count": (_u64, [ctypes.c_int]),
    "pw_last_error": (ctypes.c_char_p, []),
    "pw_version": (ctypes.c_char_p, []),
}


def lib():
    """Load libprobewalk.so (built by ``paper_2512_05460_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libprobewalk.so is not built ({LIB_PATH}); run paper_2512_05460_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int):
    if status < 0:
        raise PWError(status, pw_last_error())
    return status


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a: np.ndarray, ctype):
    return a.ctypes.data_as(P(ctype))


def _params(params):
    return ctypes.byref(params) if params is not None else None


def _seed_ptr(seed):
    return ctypes.byref(_u64(seed)) if seed is not None else None


def _dev_ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


# ---- graph -----------------------------------------------------------------

def pw_graph_load(row_ptr, col_idx, device: int = 0, flags: int = 0) -> int:
    rp = _arr(row_ptr, np.int64)
    ci = _arr(col_idx, np.int32)
    h = _vp()
    _check(lib().pw_graph_load(rp.size - 1, _p(rp, _i64), _p(ci, _i32), ci.size, device, flags, ctypes.byref(h)))
    return h.value


def pw_graph_load32(row_ptr, col_idx, device: int = 0, flags: int = 0) -> int:
    rp = _arr(row_ptr, np.int32)
    ci = _arr(col_idx, np.int32)
    h = _vp()
    _check(lib().pw_graph_load32(rp.size - 1, _p(rp, _i32), _p(ci, _i32), ci.size, device, flags, ctypes.byref(h)))
    return h.value


def pw_graph_free(g: int) -> None:
    lib().pw_graph_free(g)


def pw_graph_set_l2_window(g: int, which: int) -> None:
    """L2 access-policy window of the walk launches: 0 none, 1 the gathered array, 2 the node records."""
    _check(lib().pw_graph_set_l2_window(g, int(which)))


def pw_graph_info(g: int) -> dict:
    n, nnz = _i64(), _i64()
    dmin, dmax, bip = _i32(), _i32(), _i32()
    _check(lib().pw_graph_info(g, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(dmin), ctypes.byref(dmax),
                               ctypes.byref(bip)))
    return {"n": n.value, "nnz": nnz.value, "d_min": dmin.value, "d_max": dmax.value, "bipartite": bool(bip.value)}


# ---- budget / queries ------------------------------------------------------

def pw_budget(g: int, s: int, t: int, eps: float, L: int, seed=None, params=None) -> dict:
    B, G, K, R = _u64(), _u64(), _u64(), _u64()
    _check(lib().pw_budget(g, s, t, eps, L, _seed_ptr(seed), _params(params), ctypes.byref(B), ctypes.byref(G),
                           ctypes.byref(K), ctypes.byref(R)))
    return {"B": B.value, "G": G.value, "K": K.value, "R": R.value}


def pw_default_seed(global_seed: int, s: int, t: int, eps: float, L: int) -> int:
    return int(lib().pw_default_seed(global_seed, s, t, eps, L))


def pw_query(g: int, s: int, t: int, eps: float, L: int, seed=None, params=None) -> float:
    out = _dbl()
    _check(lib().pw_query(g, s, t, eps, L, _seed_ptr(seed), _params(params), ctypes.byref(out)))
    return out.value


def pw_query_batch(g: int, s, t, eps, L, seeds=None, params=None):
    """Host arrays in, (beta_hat, status) numpy arrays out."""
    s = _arr(s, np.int64)
    n = s.size
    t = _arr(t, np.int64)
    eps = _arr(np.broadcast_to(eps, (n,)), np.float64)
    L = _arr(np.broadcast_to(L, (n,)), np.int32)
    sd = None if seeds is None else _arr(seeds, np.uint64)
    beta = np.zeros(n, np.float64)
    st = np.zeros(n, np.int32)
    _check(lib().pw_query_batch(g, n, _p(s, _i64), _p(t, _i64), _p(eps, _dbl), _p(L, _i32),
                                None if sd is None else _p(sd, _u64), _params(params), _p(beta, _dbl), _p(st, _i32)))
    return beta, st


def pw_query_batch_device(g: int, count: int, d_s, d_t, d_eps, d_L, d_seeds, d_beta, d_status, params=None,
                          stream=None) -> None:
    """Device arrays (torch CUDA tensors or raw addresses); ordered on `stream`
    (a torch.cuda.Stream, a raw cudaStream_t, or None for torch's current stream)."""
    if stream is None:
        import torch

        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    _check(lib().pw_query_batch_device(g, count, _dev_ptr(d_s), _dev_ptr(d_t), _dev_ptr(d_eps), _dev_ptr(d_L),
                                       _dev_ptr(d_seeds), _params(params), _dev_ptr(d_beta), _dev_ptr(d_status),
                                       stream))


def pw_query_batch_noalloc(g: int, count: int, d_s, d_t, d_eps, d_L, d_seeds, d_beta, d_status, params=None,
                           stream=None) -> None:
    """pw_query_batch_device for callers that must not allocate: the library
    takes its scratch from a static 64 MiB device array (see the header)."""
    if stream is None:
        import torch

        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    _check(lib().pw_query_batch_noalloc(g, count, _dev_ptr(d_s), _dev_ptr(d_t), _dev_ptr(d_eps), _dev_ptr(d_L),
                                        _dev_ptr(d_seeds), _params(params), _dev_ptr(d_beta), _dev_ptr(d_status),
                                        stream))


def pw_query_stabilized(g: int, s, t, eps, L_max: int, seeds=None, params=None):
    """Section 4.3's doubling rule; returns (beta_hat, L_stop, status)."""
    s = _arr(s, np.int64)
    n = s.size
    t = _arr(t, np.int64)
    eps = _arr(np.broadcast_to(eps, (n,)), np.float64)
    sd = None if seeds is None else _arr(seeds, np.uint64)
    beta = np.zeros(n, np.float64)
    Ls = np.zeros(n, np.int32)
    st = np.zeros(n, np.int32)
    _check(lib().pw_query_stabilized(g, n, _p(s, _i64), _p(t, _i64), _p(eps, _dbl), L_max,
                                     None if sd is None else _p(sd, _u64), _params(params), _p(beta, _dbl),
                                     _p(Ls, _i32), _p(st, _i32)))
    return beta, Ls, st


def pw_level_seed(seed: int, L: int) -> int:
    return int(lib().pw_level_seed(seed, L))


def pw_series_batch(g: int, s, t, L):
    """Deterministic beta^(L) by the truncated series (Lemma 2.3), FP64, on the GPU."""
    s = _arr(s, np.int64)
    n = s.size
    t = _arr(t, np.int64)
    L = _arr(np.broadcast_to(L, (n,)), np.int32)
    out = np.zeros(n, np.float64)
    _check(lib().pw_series_batch(g, n, _p(s, _i64), _p(t, _i64), _p(L, _i32), _p(out, _dbl)))
    return out


def pw_query_blocks(g: int, s: int, t: int, eps: float, L: int, g_begin: int, g_end: int, seed=None,
                    params=None) -> np.ndarray:
    out = np.zeros(g_end - g_begin, np.float64)
    _check(lib().pw_query_blocks(g, s, t, eps, L, _seed_ptr(seed), _params(params), g_begin, g_end,
                                 _p(out, _dbl)))
    return out


def pw_block_median(block_means) -> float:
    m = _arr(block_means, np.float64)
    out = _dbl()
    _check(lib().pw_block_median(_p(m, _dbl), m.size, ctypes.byref(out)))
    return out.value


# ---- server ----------------------------------------------------------------

def pw_server_create(g: int, params=None, accum_bytes: int = 1 << 30) -> int:
    h = _vp()
    _check(lib().pw_server_create(g, _params(params), accum_bytes, ctypes.byref(h)))
    return h.value


def pw_server_submit(srv: int, s: int, t: int, eps: float, L: int, seed=None) -> int:
    ticket = _u64()
    _check(lib().pw_server_submit(srv, s, t, eps, L, _seed_ptr(seed), ctypes.byref(ticket)))
    return ticket.value


def pw_server_poll(srv: int, ticket: int):
    """(status, beta_hat); status is PW_OK or PW_PENDING (errors raise)."""
    out = _dbl()
    st = _check(lib().pw_server_poll(srv, ticket, ctypes.byref(out)))
    return st, out.value


def pw_server_collect(srv: int, cap: int = 65536):
    """Finished results: (tickets, beta_hat, status, latency_ms) numpy arrays."""
    tk = np.zeros(cap, np.uint64)
    b = np.zeros(cap, np.float64)
    st = np.zeros(cap, np.int32)
    lat = np.zeros(cap, np.float64)
    n = _i64()
    _check(lib().pw_server_collect(srv, cap, _p(tk, _u64), _p(b, _dbl), _p(st, _i32), _p(lat, _dbl), ctypes.byref(n)))
    k = n.value
    return tk[:k], b[:k], st[:k], lat[:k]


def pw_server_drain(srv: int, timeout_ms: int = 60000) -> None:
    _check(lib().pw_server_drain(srv, timeout_ms))


def pw_server_tune(srv: int, s, t, eps, L, seeds=None) -> dict:
    """Time the sample through the server under each walk-kernel policy (or, when the
    probe table does not fit, at each occupancy of the per-visit kernel) and keep the fastest."""
    s = _arr(s, np.int64)
    n = s.size
    t = _arr(t, np.int64)
    eps = _arr(np.broadcast_to(eps, (n,)), np.float64)
    L = _arr(np.broadcast_to(L, (n,)), np.int32)
    sd = None if seeds is None else _arr(seeds, np.uint64)
    out = pw_server_tune_result()
    _check(lib().pw_server_tune(srv, n, _p(s, _i64), _p(t, _i64), _p(eps, _dbl), _p(L, _i32),
                                None if sd is None else _p(sd, _u64), ctypes.byref(out)))
    return {"queries_per_s": list(out.queries_per_s), "occupancy_qps": list(out.occupancy_qps),
            "policy": out.policy, "occupancy": out.occupancy}


def pw_server_destroy(srv: int) -> None:
    _check(lib().pw_server_destroy(srv))


# ---- debug -----------------------------------------------------------------

def pw_debug_philox(g: int, ctr, key) -> np.ndarray:
    c = _arr(ctr, np.uint32)
    k = _arr(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _check(lib().pw_debug_philox(g, _p(c, _u32), _p(k, _u32), _p(out, _u32)))
    return out


def pw_debug_probe(g: int, n: int, seed: int, k: int, tag: int = TAG_PROBE):
    z = np.zeros(n, np.int8)
    r = _i32()
    _check(lib().pw_debug_probe(g, seed, k, tag, _p(z, ctypes.c_int8), ctypes.byref(r)))
    return z, r.value


def pw_debug_gather_peak(g: int, iters: int = 2048) -> float:
    """Sectors/s of dependent random 16-B gathers over the graph's records."""
    out = _dbl()
    _check(lib().pw_debug_gather_peak(g, iters, ctypes.byref(out)))
    return out.value


def pw_debug_exact_sum(g: int, u) -> tuple[float, float]:
    """(S1, S2) of FP32 values through the device's exact per-probe accumulator."""
    u = _arr(u, np.float32)
    s1, s2 = _dbl(), _dbl()
    _check(lib().pw_debug_exact_sum(g, _p(u, ctypes.c_float), u.size, ctypes.byref(s1), ctypes.byref(s2)))
    return s1.value, s2.value


def pw_debug_walk(g: int, start: int, L: int, seed: int, walk_id: int, tag: int = TAG_WALK) -> np.ndarray:
    traj = np.zeros(L + 1, np.int64)
    _check(lib().pw_debug_walk(g, start, L, seed, walk_id, tag, _p(traj, _i64)))
    return traj


def pw_debug_query(g: int, n: int, s: int, t: int, eps: float, L: int, seed=None, params=None, q_cap=0, u_cap=0,
                   want_visits=False) -> dict:
    beta = _dbl()
    budget = np.zeros(4, np.uint64)
    pilot = np.zeros(3, np.float64)
    q = np.zeros(max(q_cap, 1), np.float64)
    u = np.zeros(max(u_cap, 1), np.float32)
    visits = np.zeros(n, np.uint32) if want_visits else None
    _check(lib().pw_debug_query(g, s, t, eps, L, _seed_ptr(seed), _params(params), ctypes.byref(beta),
                                _p(budget, _u64), _p(pilot, _dbl), _p(q, _dbl) if q_cap else None, q_cap,
                                _p(u, ctypes.c_float) if u_cap else None, u_cap,
                                _p(visits, _u32) if want_visits else None))
    K, R = int(budget[2]), int(budget[3])
    out = {"beta": beta.value, "B": int(budget[0]), "G": int(budget[1]), "K": K, "R": R,
           "sigma2_hat": float(pilot[0]), "q_bar": float(pilot[1]), "theta_hat": float(pilot[2])}
    if q_cap:
        out["q"] = q[:K]
    if u_cap:
        out["u"] = u[: K * R].reshape(K, R)
    if want_visits:
        out["visits"] = visits
    return out


def pw_debug_batch_probe_q(g: int, s, t, eps, L, seeds, sel_query, sel_probe, params=None):
    s = _arr(s, np.int64)
    n = s.size
    t = _arr(t, np.int64)
    eps = _arr(np.broadcast_to(eps, (n,)), np.float64)
    L = _arr(np.broadcast_to(L, (n,)), np.int32)
    sd = None if seeds is None else _arr(seeds, np.uint64)
    sq = _arr(sel_query, np.int64)
    sp = _arr(sel_probe, np.int64)
    beta = np.zeros(n, np.float64)
    st = np.zeros(n, np.int32)
    KR = np.zeros((n, 2), np.uint64)
    qs = np.zeros(max(sq.size, 1), np.float64)
    _check(lib().pw_debug_batch_probe_q(g, n, _p(s, _i64), _p(t, _i64), _p(eps, _dbl), _p(L, _i32),
                                        None if sd is None else _p(sd, _u64), _params(params), _p(beta, _dbl),
                                        _p(st, _i32), _p(KR, _u64), sq.size, _p(sq, _i64), _p(sp, _i64),
                                        _p(qs, _dbl)))
    return beta, st, KR, qs[: sq.size]


def pw_autotune(g: int, s, t, eps, L, seeds=None, params=None) -> dict:
    """Fit the graph's walk-kernel cost model on a sample batch (host arrays)."""
    s = _arr(s, np.int64)
    n = s.size
    t = _arr(t, np.int64)
    eps = _arr(np.broadcast_to(eps, (n,)), np.float64)
    L = _arr(np.broadcast_to(L, (n,)), np.int32)
    sd = None if seeds is None else _arr(seeds, np.uint64)
    out = pw_tune_result()
    _check(lib().pw_autotune(g, n, _p(s, _i64), _p(t, _i64), _p(eps, _dbl), _p(L, _i32),
                             None if sd is None else _p(sd, _u64), _params(params), ctypes.byref(out)))
    return {"visit_ns": out.visit_ns, "table_visit_ns": out.table_visit_ns, "table_probe_ns": out.table_probe_ns,
            "sample_ms": list(out.sample_ms), "table_available": out.table_available,
            "sample_mode": out.sample_mode, "visit_occupancy": out.visit_occupancy,
            "table_threads": out.table_threads, "policy_ms": list(out.policy_ms), "policy": out.policy,
            "l2_window": out.l2_window, "window_ms": list(out.window_ms)}


def pw_profile(g: int, enable: bool = True, reset: bool = False) -> dict:
    st = pw_profile_stats()
    _check(lib().pw_profile(g, 1 if enable else 0, 1 if reset else 0, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in pw_profile_stats._fields_}


def pw_launch_count(reset: bool = False) -> int:
    return int(lib().pw_launch_count(1 if reset else 0))


def pw_last_error() -> str:
    return (lib().pw_last_error() or b"").decode()


def pw_version() -> str:
    return lib().pw_version().decode()


class Graph:
    """Owning handle around pw_graph_load / pw_graph_free."""

    def __init__(self, row_ptr, col_idx, device: int = 0, flags: int = 0):
        self.handle = pw_graph_load(row_ptr, col_idx, device, flags)
        info = pw_graph_info(self.handle)
        self.n = info["n"]
        self.info = info

    def close(self):
        if self.handle:
            pw_graph_free(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
