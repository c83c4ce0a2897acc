"""Graph and arrival-trace generators (inputs only, no shortest-path arithmetic).

Readings of the workload recipes:

* RNG: ``numpy.random.default_rng(seed)``; draws happen in the order written.
* Swiss roll: t ~ U[1.5*pi, 4.5*pi] (n draws), then height ~ U[0, 21] (n draws);
  point = (t cos t, height, t sin t).
* Gaussian mixture: the (components x dim) means ~ U[-10, 10] first, then labels
  uniform over the components, then N(0, sigma^2) noise.
* kNN: exact Euclidean distances in float64, self excluded, ties broken by the
  lower vertex index, symmetrised by union (an edge if either endpoint lists
  the other).
* Integer weights: max(1, rint(scale * distance)) with half-to-even rounding.
* Erdos-Renyi: each unordered pair is an edge with p = deg / (n - 1) (drawn
  as m ~ Binomial(N, p) distinct pairs out of the N pairs); a
  spanning path over a random permutation is added; weights U{1..wmax}; a
  duplicated pair keeps the smaller weight.
* Serving trace: exponential inter-arrival gaps from seed 0; request i draws its
  own n (log-uniform) and graph from seed ``first_seed + i``.

The graph problem itself (undirected, non-negative weights, distances only)
is the one of the paper's Sec. 3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Missing-edge sentinels of the library's API (0 on the diagonal, INF elsewhere
# for a non-edge).  INF32 = INT32_MAX / 2 so that any sum of two stored values
# stays below INT32_MAX; INF16 = 0x7FFF for the packed unsigned 16-bit mode.
INF32 = 1073741823
INF16 = 0x7FFF


def swiss_roll(n: int, seed: int) -> np.ndarray:
    """n points on the 3-D Swiss roll, float64, shape (n, 3)."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(1.5 * math.pi, 4.5 * math.pi, size=n)
    h = rng.uniform(0.0, 21.0, size=n)
    return np.stack([t * np.cos(t), h, t * np.sin(t)], axis=1)


def gaussian_mixture(n: int, seed: int, dim: int = 10, components: int = 8,
                     lo: float = -10.0, hi: float = 10.0, sigma: float = 1.0) -> np.ndarray:
    """n points from a mixture of isotropic Gaussians, float64, shape (n, dim)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(lo, hi, size=(components, dim))
    labels = rng.integers(0, components, size=n)
    noise = rng.normal(0.0, sigma, size=(n, dim))
    return means[labels] + noise


def knn_edges(points: np.ndarray, k: int):
    """Undirected union-kNN edge list.

    Returns (src, dst, dist) with src < dst, one entry per unordered pair,
    dist the float64 Euclidean distance.
    """
    from scipy.spatial import cKDTree

    n = points.shape[0]
    kq = min(n, k + 2)
    tree = cKDTree(points)
    dist, idx = tree.query(points, k=kq)
    dist = np.asarray(dist, dtype=np.float64).reshape(n, kq)
    idx = np.asarray(idx, dtype=np.int64).reshape(n, kq)
    rows = np.repeat(np.arange(n, dtype=np.int64), kq).reshape(n, kq)
    # order each row by (distance, index) so ties go to the lower index
    order = np.lexsort((idx, dist), axis=1)
    idx = np.take_along_axis(idx, order, axis=1)
    dist = np.take_along_axis(dist, order, axis=1)
    keep = idx != rows
    # drop self, then keep the first k survivors of every row
    rank = np.cumsum(keep, axis=1)
    keep &= rank <= k
    s = rows[keep]
    d = idx[keep]
    w = dist[keep]
    a = np.minimum(s, d)
    b = np.maximum(s, d)
    key = a * n + b
    key, first = np.unique(key, return_index=True)
    return a[first], b[first], w[first]


def int_weights(dist: np.ndarray, scale: float) -> np.ndarray:
    """max(1, rint(scale * dist)) as int64 (half-to-even rounding)."""
    return np.maximum(1, np.rint(scale * dist)).astype(np.int64)


def er_graph(n: int, seed, avg_degree: float = 16.0, wmax: int = 1000):
    """Erdos-Renyi graph plus a random spanning path; integer weights U{1..wmax}.

    ``seed`` is an int or a ``numpy.random.Generator`` to continue drawing from.
    Returns (src, dst, w) with src < dst, unique pairs (a duplicate keeps the
    smaller weight).
    """
    rng = seed if isinstance(seed, np.random.Generator) else np.random.default_rng(seed)
    p = min(1.0, avg_degree / max(1, n - 1))
    # G(n, p): the number of edges is Binomial(N, p) over the N unordered
    # pairs, and given that number the edge set is a uniform sample of pairs
    N = n * (n - 1) // 2
    m = int(rng.binomial(N, p)) if N > 0 else 0
    idx = np.sort(rng.choice(N, size=m, replace=False)).astype(np.int64) if m else np.zeros(0, np.int64)
    # pair index -> (i, j), i < j, in row-major order of the upper triangle
    start = lambda i: i * (2 * n - i - 1) // 2  # noqa: E731
    i = np.floor(((2 * n - 1) - np.sqrt((2.0 * n - 1) ** 2 - 8.0 * idx)) / 2).astype(np.int64)
    i = np.clip(i, 0, max(0, n - 2))
    for _ in range(3):
        i = np.where(start(i + 1) <= idx, i + 1, i)
        i = np.where(start(i) > idx, i - 1, i)
    s = i
    d = idx - start(i) + i + 1
    w = rng.integers(1, wmax + 1, size=s.shape[0]).astype(np.int64)
    perm = rng.permutation(n).astype(np.int64)
    ps, pd = perm[:-1], perm[1:]
    pw = rng.integers(1, wmax + 1, size=ps.shape[0]).astype(np.int64)
    s = np.concatenate([s, np.minimum(ps, pd)])
    d = np.concatenate([d, np.maximum(ps, pd)])
    w = np.concatenate([w, pw])
    key = s * n + d
    order = np.lexsort((w, key))
    key, s, d, w = key[order], s[order], d[order], w[order]
    first = np.ones(key.shape[0], dtype=bool)
    first[1:] = key[1:] != key[:-1]
    return s[first], d[first], w[first]


def dense_matrix(n: int, src, dst, w, dtype=np.int32, inf=None, ld: int | None = None,
                 directed: bool = False) -> np.ndarray:
    """Dense adjacency matrix W: 0 on the diagonal, w(i,j) on edges, INF elsewhere.

    The returned array has shape (n, ld) (ld >= n); columns n..ld-1 are
    filled with INF and are never read by the library.  A duplicated pair keeps
    the smaller weight.  ``directed=False`` mirrors every edge.
    """
    ld = n if ld is None else ld
    if inf is None:
        inf = np.inf if np.dtype(dtype).kind == "f" else INF32
    W = np.full((n, ld), inf, dtype=dtype)
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    wv = np.asarray(w).astype(dtype)
    np.minimum.at(W, (src, dst), wv)
    if not directed:
        np.minimum.at(W, (dst, src), wv)
    W[np.arange(n), np.arange(n)] = 0
    return W


@dataclass
class Graph:
    name: str
    n: int
    src: np.ndarray
    dst: np.ndarray
    w: np.ndarray          # int64 weights, or float64 for the fp32 variant
    dtype: str             # "int32", "fp32" or "u16"


def serving_trace(num: int = 2000, rate: float = 200.0, seed: int = 0,
                  first_seed: int = 1000, n_lo: int = 128, n_hi: int = 4096):
    """Poisson arrival trace.  Returns (arrival_s, n, seeds) numpy arrays.

    Arrival gaps ~ Exp(mean 1/rate) from ``seed``; request i takes
    n = round(exp(U[ln n_lo, ln n_hi])) from its own seed ``first_seed + i``.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=num)
    arrival = np.cumsum(gaps) - gaps[0]
    seeds = np.arange(first_seed, first_seed + num, dtype=np.int64)
    ns = np.empty(num, dtype=np.int64)
    for i, s in enumerate(seeds):
        r = np.random.default_rng(int(s))
        ns[i] = int(round(math.exp(r.uniform(math.log(n_lo), math.log(n_hi)))))
    return arrival, ns, seeds


def serving_request(seed: int, n_lo: int = 128, n_hi: int = 4096, wmax: int = 1000):
    """The ER graph of one serving request (same n as ``serving_trace``)."""
    r = np.random.default_rng(int(seed))
    n = int(round(math.exp(r.uniform(math.log(n_lo), math.log(n_hi)))))
    s, d, w = er_graph(n, r, avg_degree=16.0, wmax=wmax)
    return Graph(f"er-{seed}", n, s, d, w, "int32")


# name -> (builder) for the five workloads; every builder is deterministic.
def _knn_roll(n, seed, k, scale):
    pts = swiss_roll(n, seed)
    s, d, dist = knn_edges(pts, k)
    return s, d, int_weights(dist, scale)


def _knn_gmm(n, seed, k, scale):
    pts = gaussian_mixture(n, seed)
    s, d, dist = knn_edges(pts, k)
    if scale is None:
        return s, d, dist
    return s, d, int_weights(dist, scale)


WORKLOADS = {
    # n=512 Swiss roll, k=8, weights max(1, rint(100 d)), int32
    "roll512": lambda: Graph("roll512", 512, *_knn_roll(512, 0, 8, 100.0), "int32"),
    # n=16384 10-D Gaussian mixture, k=10, weights max(1, rint(50 d)), int32
    "gmm16k": lambda: Graph("gmm16k", 16384, *_knn_gmm(16384, 1, 10, 50.0), "int32"),
    # same points, raw Euclidean fp32 weights
    "gmm16k_f32": lambda: Graph("gmm16k_f32", 16384, *_knn_gmm(16384, 1, 10, None), "fp32"),
    # n=65536 Swiss roll, k=10, weights max(1, rint(4 d)); int32 and packed u16
    "roll64k": lambda: Graph("roll64k", 65536, *_knn_roll(65536, 2, 10, 4.0), "int32"),
    # n=262144 Swiss roll, k=10, weights max(1, rint(2 d)); packed u16 in place
    "roll256k": lambda: Graph("roll256k", 262144, *_knn_roll(262144, 3, 10, 2.0), "u16"),
}


def workload(name: str) -> Graph:
    return WORKLOADS[name]()
