"""Exact and truncated-series biharmonic distance, FP64 (ORACLE, test infrastructure only).

* :func:`exact_beta` — Definition 2.1 (Eq. exact): beta(s,t) = b^T L^{2+} b with
  L^+ = (L + 11^T/n)^{-1} - 11^T/n (Section 2.1).  Dense LU inverse; n up to a
  few thousand.
* :func:`series_beta` — Lemma 2.3 (Eq. tr-beta-exp-Liu): h^(L) = sum_{i<=L}
  P^i D^{-1} b_st, beta^(L) = ||h||^2 - (1^T h)^2 / n, by L sparse matvecs.
* :func:`series_h` — the vector h^(L) itself (used by the probe identity of
  Lemma 3.3 and the walk identity of Eq. phi-rw-identity).
* :func:`mixing_lambda` — lambda = max(|lambda_2|, |lambda_n|) of P (Section 2.1),
  dense eigenvalues for small graphs.
* :func:`truncation_length` — Eq. uni_l.
* :func:`effective_resistance` — R_eff(s,t) = b^T L^+ b (proof of Lemma 3.5).
"""

from __future__ import annotations

import math

import numpy as np


def _adjacency(row_ptr, col_idx, n):
    a = np.zeros((n, n), dtype=np.float64)
    src = np.repeat(np.arange(n), np.diff(row_ptr))
    a[src, col_idx] = 1.0
    return a


def laplacian_pinv(row_ptr, col_idx, n: int) -> np.ndarray:
    """L^+ = (L + J/n)^{-1} - J/n (Section 2.1)."""
    a = _adjacency(row_ptr, col_idx, n)
    lap = np.diag(a.sum(axis=1)) - a
    j = np.full((n, n), 1.0 / n)
    return np.linalg.inv(lap + j) - j


def exact_beta_matrix(row_ptr, col_idx, n: int) -> np.ndarray:
    """All-pairs beta(s,t) = L2_ss + L2_tt - 2 L2_st with L2 = L^+ L^+ (Eq. exact)."""
    lp = laplacian_pinv(row_ptr, col_idx, n)
    l2 = lp @ lp
    dg = np.diag(l2)
    return dg[:, None] + dg[None, :] - 2.0 * l2


def exact_beta(row_ptr, col_idx, n: int, s: int, t: int) -> float:
    """beta(s,t) = ||L^+ (e_s - e_t)||^2 (Eq. exact)."""
    lp = laplacian_pinv(row_ptr, col_idx, n)
    x = lp[:, s] - lp[:, t]
    return float(x @ x)


def effective_resistance(row_ptr, col_idx, n: int, s: int, t: int) -> float:
    lp = laplacian_pinv(row_ptr, col_idx, n)
    return float(lp[s, s] + lp[t, t] - 2.0 * lp[s, t])


def _neumaier(values: np.ndarray) -> float:
    total = 0.0
    comp = 0.0
    for v in values.tolist():
        t = total + v
        if abs(total) >= abs(v):
            comp += (total - t) + v
        else:
            comp += (v - t) + total
        total = t
    return total + comp


def series_h(row_ptr, col_idx, n: int, s: int, t: int, L: int) -> np.ndarray:
    """h^(L) = sum_{i=0}^{L} P^i D^{-1} b_st with P = D^{-1} A (Lemma 2.3)."""
    from scipy.sparse import csr_matrix

    deg = np.diff(row_ptr).astype(np.float64)
    a = csr_matrix((np.ones(len(col_idx)), col_idx, row_ptr), shape=(n, n))
    x = np.zeros(n)
    x[s] += 1.0 / deg[s]
    x[t] -= 1.0 / deg[t]
    h = np.zeros(n)
    for _ in range(L):
        h += x
        x = (a @ x) / deg  # (P x)_i = (1/d_i) sum_{j in N(i)} x_j
    h += x
    return h


def series_beta(row_ptr, col_idx, n: int, s: int, t: int, L: int) -> float:
    """beta^(L)(s,t) = ||h^(L)||^2 - (1^T h^(L))^2 / n (Eq. tr-beta-exp-Liu), FP64
    with compensated sums."""
    h = series_h(row_ptr, col_idx, n, s, t, L)
    sq = _neumaier(h * h)
    tot = _neumaier(h)
    return sq - tot * tot / n


def series_beta_many(row_ptr, col_idx, n: int, s, t, L: int) -> np.ndarray:
    """beta^(L) for many pairs at once (columns of a sparse matrix power series)."""
    from scipy.sparse import csr_matrix

    s = np.asarray(s, dtype=np.int64)
    t = np.asarray(t, dtype=np.int64)
    q = s.size
    deg = np.diff(row_ptr).astype(np.float64)
    a = csr_matrix((np.ones(len(col_idx)), col_idx, row_ptr), shape=(n, n))
    x = np.zeros((n, q))
    cols = np.arange(q)
    x[s, cols] += 1.0 / deg[s]
    x[t, cols] -= 1.0 / deg[t]
    h = np.zeros((n, q))
    for _ in range(L):
        h += x
        x = (a @ x) / deg[:, None]
    h += x
    out = np.empty(q)
    for j in range(q):
        col = h[:, j]
        sq = math.fsum((col * col).tolist())
        tot = math.fsum(col.tolist())
        out[j] = sq - tot * tot / n
    return out


def mixing_lambda(row_ptr, col_idx, n: int) -> float:
    """lambda = max(|lambda_2|, |lambda_n|) of P = D^{-1} A (Section 2.1), computed
    from the symmetric matrix D^{-1/2} A D^{-1/2}, which has the same spectrum."""
    a = _adjacency(row_ptr, col_idx, n)
    dinv = 1.0 / np.sqrt(a.sum(axis=1))
    ev = np.linalg.eigvalsh(dinv[:, None] * a * dinv[None, :])
    ev = np.sort(ev)[::-1]
    return float(max(abs(ev[1]), abs(ev[-1])))


def truncation_length(n: int, lam: float, eta: float) -> int:
    """Eq. uni_l: L = ceil(log(12 n / (eta (1 - lambda)^2)) / log(1 / lambda))."""
    return int(math.ceil(math.log(12.0 * n / (eta * (1.0 - lam) ** 2)) / math.log(1.0 / lam)))
