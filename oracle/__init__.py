"""ProbeWalk ORACLE — test infrastructure only.

Plain, slow, obviously correct CPU restatement of what the GPU path computes:

* :mod:`oracle.exact` — exact beta from the dense FP64 pseudoinverse
  (Definition 2.1, Section 2.1) and the L-truncated series (Lemma 2.3).
* ``walker.c`` (loaded here through ctypes) — Philox4x32-10, the stateless
  Paired-Sign Probe generator (Section 3.3), the serial Algorithm 1 walker with
  its U-statistic and median-of-means, and the budgets.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA path and never
imports it; the product path never imports this.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import exact  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle.so")
_SRC = os.path.join(_HERE, "walker.c")
_lock = threading.Lock()
_lib = None

MODE_PILOT, MODE_THEORY, MODE_SCALED, MODE_FIXED, MODE_ADAPTIVE = 0, 1, 2, 3, 4
TAG_WALK, TAG_WALK_PILOT, TAG_PROBE, TAG_PROBE_PILOT = 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile walker.c with gcc (no fused multiply-add, no fast-math, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIBPATH) and os.path.getmtime(_LIBPATH) >= os.path.getmtime(_SRC):
        return _LIBPATH
    tmp = _LIBPATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


class BudgetCfg(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32),
        ("K0", ctypes.c_int32),
        ("R0", ctypes.c_int32),
        ("delta", ctypes.c_double),
        ("c_B", ctypes.c_double),
        ("c_R", ctypes.c_double),
        ("B", ctypes.c_uint64),
        ("G", ctypes.c_uint64),
        ("R", ctypes.c_uint64),
        ("R_max", ctypes.c_uint64),
        ("z", ctypes.c_double),
        ("cap", ctypes.c_double),
    ]


def budget_cfg(mode=MODE_PILOT, delta=0.01, c_B=0.0, c_R=0.0, B=0, G=0, R=0, R_max=0, K0=0, R0=0,
               z=0.0, cap=0.0) -> BudgetCfg:
    return BudgetCfg(mode, K0, R0, delta, c_B, c_R, B, G, R, R_max, z, cap)


def _configure(L):
    P = ctypes.POINTER
    u32p, u64p, i64p, i32p = P(ctypes.c_uint32), P(ctypes.c_uint64), P(ctypes.c_int64), P(ctypes.c_int32)
    dp, fp, i8p = P(ctypes.c_double), P(ctypes.c_float), P(ctypes.c_int8)
    L.orc_philox.argtypes = [u32p, u32p, u32p]
    L.orc_philox.restype = None
    L.orc_default_seed.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_int32]
    L.orc_default_seed.restype = ctypes.c_uint64
    L.orc_probe_vector.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, i8p, u64p]
    L.orc_probe_vector.restype = ctypes.c_int
    L.orc_walk.argtypes = [i64p, i32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64,
                           ctypes.c_uint32, i64p]
    L.orc_walk.restype = ctypes.c_int
    L.orc_query.argtypes = [i64p, i32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                            ctypes.c_int32, ctypes.c_uint64, P(BudgetCfg), dp, u64p, dp, dp, fp, u32p]
    L.orc_query.restype = ctypes.c_int
    L.orc_budget_query.argtypes = [i64p, i32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                   ctypes.c_int32, ctypes.c_uint64, P(BudgetCfg), u64p, dp]
    L.orc_budget_query.restype = ctypes.c_int
    L.orc_probe_q.argtypes = [i64p, i32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                              ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, u32p, dp]
    L.orc_probe_q.restype = ctypes.c_int
    L.orc_query_many.argtypes = [i64p, i32p, ctypes.c_int64, ctypes.c_int64, i64p, i64p, dp, i32p, u64p,
                                 P(BudgetCfg), ctypes.c_int, dp, u64p, i32p]
    L.orc_query_many.restype = ctypes.c_int
    L.orc_level_seed.argtypes = [ctypes.c_uint64, ctypes.c_int32]
    L.orc_level_seed.restype = ctypes.c_uint64
    L.orc_median_of_means.argtypes = [dp, ctypes.c_uint64, ctypes.c_uint64]
    L.orc_median_of_means.restype = ctypes.c_double
    L.orc_pilot_u.argtypes = [i64p, i32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                              ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, fp]
    L.orc_pilot_u.restype = ctypes.c_int
    L.orc_adaptive_B.argtypes = [dp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.orc_adaptive_B.restype = ctypes.c_uint64
    L.orc_exact_sum_f32.argtypes = [fp, ctypes.c_int64, ctypes.c_int]
    L.orc_exact_sum_f32.restype = ctypes.c_double
    L.orc_max_threads.argtypes = []
    L.orc_max_threads.restype = ctypes.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(ctypes.CDLL(_LIBPATH))
    return _lib


def build_variant(source_text: str, out_dir: str) -> str:
    """Compile an edited copy of walker.c (used by the tests that plant
    mistakes in the oracle to show that its pins catch them)."""
    src = os.path.join(out_dir, "walker_variant.c")
    so = os.path.join(out_dir, "liboracle_variant.so")
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", so, src,
                    "-lm"], check=True)
    return so


class use_variant:
    """Context manager that routes this module's wrappers to a compiled variant."""

    def __init__(self, so_path: str):
        self.so_path = so_path

    def __enter__(self):
        global _lib
        lib()
        self._saved = _lib
        _lib = _configure(ctypes.CDLL(self.so_path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    return rp, ci


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def default_seed(global_seed: int, s: int, t: int, eps: float, L: int) -> int:
    return int(lib().orc_default_seed(global_seed, s, t, eps, L))


def probe_vector(n: int, seed: int, k: int, tag: int = TAG_PROBE):
    """(z, pi, r) for probe k of the query keyed by `seed`."""
    z = np.zeros(n, np.int8)
    pi = np.zeros(n, np.uint64)
    r = lib().orc_probe_vector(n, seed, k, tag, _ptr(z, ctypes.c_int8), _ptr(pi, ctypes.c_uint64))
    if r < 0:
        raise ValueError("invalid probe arguments")
    return z, pi, r


def walk(g, start: int, L: int, seed: int, walk_id: int, tag: int = TAG_WALK) -> np.ndarray:
    rp, ci = _csr(g)
    traj = np.zeros(L + 1, np.int64)
    lib().orc_walk(_ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), start, L, seed, walk_id, tag,
                   _ptr(traj, ctypes.c_int64))
    return traj


def query(g, s: int, t: int, eps: float, L: int, seed: int, cfg: BudgetCfg | None = None, want_q=False,
          want_u=False, want_visits=False) -> dict:
    """Algorithm 1 for one query; returns beta_hat, budget (B, G, K, R), pilot
    diagnostics, and optionally Q_R per probe, U_p per replica, visit counts."""
    cfg = cfg or budget_cfg()
    rp, ci = _csr(g)
    L_ = lib()
    budget = np.zeros(4, np.uint64)
    pilot = np.zeros(3, np.float64)
    beta = ctypes.c_double(0.0)
    if s != t and (want_q or want_u):
        if L_.orc_budget_query(_ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), g.n, s, t, eps, L, seed,
                               ctypes.byref(cfg), _ptr(budget, ctypes.c_uint64), _ptr(pilot, ctypes.c_double)) != 0:
            raise ValueError("invalid query")
    K = int(budget[2])
    R = int(budget[3])
    q = np.zeros(max(K, 1), np.float64) if want_q else None
    u = np.zeros(max(K * R, 1), np.float32) if want_u else None
    visits = np.zeros(g.n, np.uint32) if want_visits else None
    rc = L_.orc_query(_ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), g.n, s, t, eps, L, seed, ctypes.byref(cfg),
                      ctypes.byref(beta), _ptr(budget, ctypes.c_uint64), _ptr(pilot, ctypes.c_double),
                      None if q is None else _ptr(q, ctypes.c_double),
                      None if u is None else _ptr(u, ctypes.c_float),
                      None if visits is None else _ptr(visits, ctypes.c_uint32))
    if rc != 0:
        raise ValueError("invalid query")
    K = int(budget[2])
    R = int(budget[3])
    out = {"beta": beta.value, "B": int(budget[0]), "G": int(budget[1]), "K": K, "R": R,
           "sigma2_hat": float(pilot[0]), "q_bar": float(pilot[1]), "theta_hat": float(pilot[2])}
    if want_q:
        out["q"] = q[:K]
    if want_u:
        out["u"] = u[: K * R].reshape(K, R)
    if want_visits:
        out["visits"] = visits
    return out


def budget(g, s: int, t: int, eps: float, L: int, seed: int, cfg: BudgetCfg | None = None) -> dict:
    cfg = cfg or budget_cfg()
    rp, ci = _csr(g)
    b = np.zeros(4, np.uint64)
    pilot = np.zeros(3, np.float64)
    if lib().orc_budget_query(_ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), g.n, s, t, eps, L, seed,
                              ctypes.byref(cfg), _ptr(b, ctypes.c_uint64), _ptr(pilot, ctypes.c_double)) != 0:
        raise ValueError("invalid query")
    return {"B": int(b[0]), "G": int(b[1]), "K": int(b[2]), "R": int(b[3]), "sigma2_hat": float(pilot[0]),
            "q_bar": float(pilot[1]), "theta_hat": float(pilot[2])}


def probe_q(g, s: int, t: int, L: int, seed: int, R: int, ks) -> np.ndarray:
    rp, ci = _csr(g)
    ks = np.ascontiguousarray(ks, dtype=np.uint32)
    out = np.zeros(ks.size, np.float64)
    lib().orc_probe_q(_ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), g.n, s, t, L, seed, R, ks.size,
                      _ptr(ks, ctypes.c_uint32), _ptr(out, ctypes.c_double))
    return out


def query_many(g, s, t, eps, L, seeds, cfg: BudgetCfg | None = None, threads: int = 0):
    """Independent queries, one OpenMP thread per query; returns (beta, budgets[count,4], status)."""
    cfg = cfg or budget_cfg()
    rp, ci = _csr(g)
    s = np.ascontiguousarray(s, dtype=np.int64)
    count = s.size
    t = np.ascontiguousarray(t, dtype=np.int64)
    eps = np.ascontiguousarray(np.broadcast_to(eps, (count,)), dtype=np.float64)
    L = np.ascontiguousarray(np.broadcast_to(L, (count,)), dtype=np.int32)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    beta = np.zeros(count, np.float64)
    budgets = np.zeros((count, 4), np.uint64)
    status = np.zeros(count, np.int32)
    lib().orc_query_many(_ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), g.n, count, _ptr(s, ctypes.c_int64),
                         _ptr(t, ctypes.c_int64), _ptr(eps, ctypes.c_double), _ptr(L, ctypes.c_int32),
                         _ptr(seeds, ctypes.c_uint64), ctypes.byref(cfg), threads, _ptr(beta, ctypes.c_double),
                         _ptr(budgets, ctypes.c_uint64), _ptr(status, ctypes.c_int32))
    return beta, budgets, status


def level_seed(seed: int, L: int) -> int:
    return int(lib().orc_level_seed(seed, L))


def stabilized(g, s: int, t: int, eps: float, L_max: int, seed: int, cfg: BudgetCfg | None = None):
    """The stabilization rule of Section 4.3: from L = 1, double L (capped at
    L_max) and accept L_stop = 2L once |beta(2L) - beta(L)| <= (eps/2)|beta(2L)|;
    each level is an independent run of Algorithm 1 with seed level_seed(seed, L).
    Returns (beta_hat, L_stop, per-level estimates)."""
    if s == t:
        return 0.0, 1, {}
    levels = {}
    L = 1
    prev = None
    while True:
        cur = query(g, s, t, eps, L, level_seed(seed, L), cfg)["beta"]
        levels[L] = cur
        if prev is not None and abs(cur - prev) <= eps / 2 * abs(cur):
            return cur, L, levels
        if L >= L_max:
            return cur, L, levels
        prev = cur
        L = min(2 * L, L_max)


def exact_sum_f32(u, square: bool = False) -> float:
    """The oracle's S1 (or S2 with square=True) of FP32 values: the exact sum
    rounded once to the nearest double."""
    u = np.ascontiguousarray(u, dtype=np.float32)
    return float(lib().orc_exact_sum_f32(_ptr(u, ctypes.c_float), u.size, 1 if square else 0))


def adaptive_B(q, B1: int, B: int, G: int, eps: float, z: float, d_s: float, d_t: float) -> int:
    """The ADAPTIVE budget's B* from first-stage values q[0 .. G*B1)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    if q.size < G * B1:
        raise ValueError("q holds fewer than G*B1 values")
    return int(lib().orc_adaptive_B(_ptr(q, ctypes.c_double), B1, B, G, eps, z, d_s, d_t))


def median_of_means(q, B: int, G: int) -> float:
    """Median of the G means of B contiguous values of q (Eq. final-estimator)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    if q.size < B * G:
        raise ValueError("q holds fewer than B*G values")
    return float(lib().orc_median_of_means(_ptr(q, ctypes.c_double), B, G))


def pilot_u(g, s: int, t: int, L: int, seed: int, K0: int = 64, R0: int = 32) -> np.ndarray:
    """U_p of the PILOT stage (K0 probes x R0 replicas on the pilot streams), shape (K0, R0)."""
    rp, ci = _csr(g)
    u = np.zeros(K0 * R0, np.float32)
    if lib().orc_pilot_u(_ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), g.n, s, t, L, seed, K0, R0,
                         _ptr(u, ctypes.c_float)) != 0:
        raise ValueError("invalid pilot arguments")
    return u.reshape(K0, R0)


def max_threads() -> int:
    return int(lib().orc_max_threads())
