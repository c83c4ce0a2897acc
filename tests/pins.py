"""Independent routes to the shortest-path metric, used to pin the oracle.

None of these shares code with ``oracle/``:

* ``brute_force``      enumerate every simple path (tiny n only)
* ``repeated_squaring`` the paper's Alg. 1 route: D <- min(D, D (x) D), about
                        log2(n) times, written with numpy broadcasting
* ``rank1_fw``         the paper's Alg. 2 route: for every k, the rank-1 update
                        of Table 1 FloydWarshallUpdate, C = col_k 1^T + 1 row_k,
                        then MatMin
"""
import math

import numpy as np

INF = 1073741823


def brute_force(n, edges, directed=False):
    """edges: iterable of (u, v, w).  Returns an (n, n) int64 matrix, INF for no path."""
    adj = [dict() for _ in range(n)]
    for u, v, w in edges:
        if v not in adj[u] or w < adj[u][v]:
            adj[u][v] = w
        if not directed and (u not in adj[v] or w < adj[v][u]):
            adj[v][u] = w
    D = np.full((n, n), INF, dtype=np.int64)
    for s in range(n):
        D[s, s] = 0
        stack = [(s, 0, 1 << s)]
        while stack:
            u, dist, seen = stack.pop()
            for v, w in adj[u].items():
                if seen & (1 << v):
                    continue
                nd = dist + w
                if nd < D[s, v]:
                    D[s, v] = nd
                stack.append((v, nd, seen | (1 << v)))
    return D


def _minplus_square(D):
    """(D (x) D)_ij = min_t D_it + D_tj with INF absorbing."""
    big = D.astype(np.float64)
    big[D >= INF] = np.inf
    out = np.min(big[:, :, None] + big[None, :, :], axis=1)
    res = np.where(np.isinf(out), INF, out).astype(np.int64)
    return np.minimum(D, res)


def repeated_squaring(W):
    """Alg. 1 route: about ceil(log2(n)) min-plus squarings of W (0 on the diagonal)."""
    D = np.asarray(W, dtype=np.int64).copy()
    n = D.shape[0]
    for _ in range(max(1, math.ceil(math.log2(max(2, n))))):
        D = _minplus_square(D)
    return D


def rank1_fw(W):
    """Alg. 2 route: per-k rank-1 update C = D[:,k] 1^T + 1 D[k,:], then MatMin."""
    D = np.asarray(W, dtype=np.int64).copy()
    n = D.shape[0]
    for k in range(n):
        col = D[:, k][:, None]
        row = D[k, :][None, :]
        C = col + row
        C[(col >= INF) | (row >= INF)] = INF
        D = np.minimum(D, C)
    return D


def random_graph(rng, n, p, wmax, directed=False, zero_ok=False):
    edges = []
    for u in range(n):
        for v in range(n):
            if u == v or (not directed and v <= u):
                continue
            if rng.random() < p:
                lo = 0 if zero_ok else 1
                edges.append((u, v, int(rng.integers(lo, wmax + 1))))
    return edges


def dense(n, edges, directed=False, dtype=np.int64):
    W = np.full((n, n), INF, dtype=dtype)
    for u, v, w in edges:
        W[u, v] = min(W[u, v], w)
        if not directed:
            W[v, u] = min(W[v, u], w)
    np.fill_diagonal(W, 0)
    return W
