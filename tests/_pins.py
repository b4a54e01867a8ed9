"""Independent numpy checks used to pin the oracle (test helpers).

Nothing here calls the oracle or the CUDA path: each function restates a
mathematical fact about the FCLS problem of Sec. 2.2-2.3 (whitened least
squares with x >= 0 and sum x = 1) with plain numpy/LAPACK calls.
"""
from __future__ import annotations

import itertools

import numpy as np


def whiten(S, sigma):
    """G = S W^2 S^T and B = W^2 S with W = diag(1/sigma) (Sec. 2.3)."""
    S = np.asarray(S, dtype=np.float64)
    w2 = 1.0 / np.asarray(sigma, dtype=np.float64) ** 2
    B = S * w2[None, :]
    return B @ S.T, B


def qp_terms(S, sigma, y):
    G, B = whiten(S, sigma)
    y = np.asarray(y, dtype=np.float64)
    c = B @ y
    s = float(np.sum(y * y / np.asarray(sigma, dtype=np.float64) ** 2))
    return G, c, s


def objective(G, c, s, x):
    return 0.5 * x @ G @ x - c @ x + 0.5 * s


def eq_constrained(G, c, idx):
    """Minimiser of 1/2 x'Gx - c'x on {x_i = 0 off idx, sum x = 1} (SCLS on
    the support, Sec. 2.2) via the bordered KKT system; None if singular."""
    k = len(idx)
    K = np.zeros((k + 1, k + 1))
    K[:k, :k] = G[np.ix_(idx, idx)]
    K[:k, k] = 1.0
    K[k, :k] = 1.0
    rhs = np.concatenate([c[list(idx)], [1.0]])
    try:
        sol = np.linalg.solve(K, rhs)
    except np.linalg.LinAlgError:
        return None
    if not np.all(np.isfinite(sol)):
        return None
    x = np.zeros(G.shape[0])
    x[list(idx)] = sol[:k]
    return x


def brute_force(G, c, s=0.0):
    """Enumerate every support (the exhaustive-combination procedure of
    Sec. 2.1, used here as a check): keep the feasible minimum."""
    P = G.shape[0]
    best, best_f = None, np.inf
    for k in range(1, P + 1):
        for idx in itertools.combinations(range(P), k):
            x = eq_constrained(G, c, idx)
            if x is None or np.any(x < -1e-12):
                continue
            f = objective(G, c, s, np.maximum(x, 0.0))
            if f < best_f - 1e-13 * max(1.0, abs(f)):
                best, best_f = np.maximum(x, 0.0), f
    return best


def fw_gap(G, c, x):
    """Frank-Wolfe gap g'x - min_i g_i, g = Gx - c: an upper bound on
    f(x) - f* over the simplex for any feasible x (convexity)."""
    g = G @ x - c
    return float(g @ x - g.min())


def kkt_violation(G, c, x, support_tol):
    """Max KKT violation of a feasible x: with nu = -mean(g_S) on the
    support S = {x_i > support_tol}, returns (max |g_S + nu|,
    max(-(g_i + nu)) off S)."""
    g = G @ x - c
    S = x > support_tol
    nu = -np.mean(g[S])
    stat = float(np.max(np.abs(g[S] + nu)))
    dual = float(np.max(-(g[~S] + nu))) if np.any(~S) else 0.0
    return stat, dual


def support_sigma(G, idx):
    """sqrt diag of the top-left block of [[G_SS, 1],[1^T, 0]]^-1 on idx."""
    k = len(idx)
    K = np.zeros((k + 1, k + 1))
    K[:k, :k] = G[np.ix_(idx, idx)]
    K[:k, k] = 1.0
    K[k, :k] = 1.0
    Ki = np.linalg.inv(K)
    sx = np.zeros(G.shape[0])
    sx[list(idx)] = np.sqrt(np.maximum(np.diag(Ki)[:k], 0.0))
    return sx
