"""CPU oracle for all-pairs shortest paths -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  The CUDA
library (``paper_1902_04446_gb300``) never imports it and shares no code with
it; the two meet only at the seeded inputs from ``gen``.

What it computes is the plain definition from the paper's Sec. 3: for an
undirected graph with non-negative weights, the shortest-path length between
every pair of vertices (no paths); 0 on the diagonal; INF exactly on pairs in
different components.  The blocked algorithm of Sec. 4.4/4.5 reaches this
exact result for integer weights in any relaxation order, so the oracle is the
definition, not the blocked algorithm:

* ``fw``            textbook Floyd-Warshall in int64 / float64 (C, single thread)
* ``dijkstra``      binary-heap Dijkstra from a list of sources (C, threads)
* ``minplus``       C = min(C, A (x) B), Table 1 MatProd followed by MatMin
* ``components``    union-find connected components
* ``int16_bound``   the packed-16-bit enable test: per component, twice the
                    eccentricity of one vertex, compared with INF16
* ``pack_u16`` / ``unpack_u16``  the int32 <-> unsigned 16-bit storage maps

Pins (what ties these to something other than themselves) live in
``tests/test_oracle_pins.py``: brute-force path enumeration, closed forms,
invariants, independent routes (repeated min-plus squaring, Alg. 1; per-k
rank-1 updates, Alg. 2) and SciPy's csgraph routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apsp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# sentinels used by the oracle (the same numeric conventions as the library's
# API, restated here so that the oracle does not import the library)
INF32 = 1073741823
INF16 = 0x7FFF


def build(force: bool = False) -> str:
    """Compile ``apsp_oracle.c`` into ``liboracle.so`` with gcc (plain C99)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-shared", "-fPIC",
               "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64p = ctypes.POINTER(ctypes.c_int64)
            f64p = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.oracle_fw_i64.argtypes = [i64p, i64, i64, i64, i64]
            lib.oracle_fw_f64.argtypes = [f64p, i64, i64, i64]
            lib.oracle_minplus_i64.argtypes = [i64p, i64p, i64p, i64, i64, i64, i64]
            lib.oracle_minplus_f64.argtypes = [f64p, f64p, f64p, i64, i64, i64]
            lib.oracle_dijkstra_i64.argtypes = [i64, i64p, i64p, i64p, i64p, i64, i64p, i64, ctypes.c_int]
            lib.oracle_dijkstra_f64.argtypes = [i64, i64p, i64p, f64p, i64p, i64, f64p, ctypes.c_int]
            for f in ("oracle_fw_i64", "oracle_fw_f64", "oracle_minplus_i64", "oracle_minplus_f64",
                      "oracle_dijkstra_i64", "oracle_dijkstra_f64"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def fw(W: np.ndarray, k_begin: int = 0, k_end: int | None = None) -> np.ndarray:
    """Floyd-Warshall on a dense square matrix (Sec. 3; Table 1 FloydWarshall).

    Integer input is solved in int64 with INF32 as the "no path" sentinel;
    floating input in float64 with +inf.  ``k_begin``/``k_end`` restrict the
    outer loop (a full solve is 0..n); the benchmark times a bounded slice.
    """
    lib = _load()
    W = np.asarray(W)
    n = W.shape[0]
    assert W.ndim == 2 and W.shape[1] >= n
    k_end = n if k_end is None else k_end
    if W.dtype.kind == "f":
        d = np.ascontiguousarray(W[:, :n], dtype=np.float64).copy()
        rc = lib.oracle_fw_f64(_p(d, ctypes.c_double), n, k_begin, k_end)
    else:
        d = np.ascontiguousarray(W[:, :n], dtype=np.int64).copy()
        rc = lib.oracle_fw_i64(_p(d, ctypes.c_int64), n, INF32, k_begin, k_end)
    if rc != 0:
        raise ValueError("oracle fw: bad arguments")
    return d


def minplus(A: np.ndarray, B: np.ndarray, C: np.ndarray) -> np.ndarray:
    """min(C, A (x) B) with (A (x) B)_ij = min_t A_it + B_tj (Table 1 MatProd + MatMin)."""
    lib = _load()
    m, kk = A.shape
    kk2, nn = B.shape
    assert kk == kk2 and C.shape == (m, nn)
    if A.dtype.kind == "f":
        a = np.ascontiguousarray(A, dtype=np.float64)
        b = np.ascontiguousarray(B, dtype=np.float64)
        c = np.ascontiguousarray(C, dtype=np.float64).copy()
        rc = lib.oracle_minplus_f64(_p(a, ctypes.c_double), _p(b, ctypes.c_double), _p(c, ctypes.c_double), m, kk, nn)
    else:
        a = np.ascontiguousarray(A, dtype=np.int64)
        b = np.ascontiguousarray(B, dtype=np.int64)
        c = np.ascontiguousarray(C, dtype=np.int64).copy()
        rc = lib.oracle_minplus_i64(_p(a, ctypes.c_int64), _p(b, ctypes.c_int64), _p(c, ctypes.c_int64),
                                    m, kk, nn, INF32)
    if rc != 0:
        raise ValueError("oracle minplus: bad arguments")
    return c


def csr(n: int, src, dst, w, directed: bool = False):
    """CSR adjacency (both directions of every undirected edge)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = np.asarray(w)
    if not directed:
        src, dst, w = np.concatenate([src, dst]), np.concatenate([dst, src]), np.concatenate([w, w])
    order = np.argsort(src, kind="stable")
    col = np.ascontiguousarray(dst[order])
    ww = np.ascontiguousarray(w[order])
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, src + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, col, ww


def dijkstra(n: int, src, dst, w, sources, threads: int | None = None, directed: bool = False) -> np.ndarray:
    """Rows of the distance matrix for the given sources (binary-heap Dijkstra).

    Integer weights give int64 rows with INF32 for unreachable vertices;
    float weights give float64 rows with +inf.
    """
    lib = _load()
    rowptr, col, ww = csr(n, src, dst, w, directed)
    sources = np.ascontiguousarray(np.asarray(sources, dtype=np.int64))
    threads = threads or max(1, min(os.cpu_count() or 1, 64))
    if np.asarray(w).dtype.kind == "f":
        wd = np.ascontiguousarray(ww, dtype=np.float64)
        out = np.empty((sources.shape[0], n), dtype=np.float64)
        rc = lib.oracle_dijkstra_f64(n, _p(rowptr, ctypes.c_int64), _p(col, ctypes.c_int64), _p(wd, ctypes.c_double),
                                     _p(sources, ctypes.c_int64), sources.shape[0], _p(out, ctypes.c_double), threads)
    else:
        wi = np.ascontiguousarray(ww, dtype=np.int64)
        if wi.size and wi.min() < 0:
            raise ValueError("negative weight: an undirected negative edge is a negative cycle (Sec. 3)")
        out = np.empty((sources.shape[0], n), dtype=np.int64)
        rc = lib.oracle_dijkstra_i64(n, _p(rowptr, ctypes.c_int64), _p(col, ctypes.c_int64), _p(wi, ctypes.c_int64),
                                     _p(sources, ctypes.c_int64), sources.shape[0], _p(out, ctypes.c_int64), INF32,
                                     threads)
    if rc != 0:
        raise ValueError("oracle dijkstra: bad arguments or out of memory")
    return out


def components(n: int, src, dst) -> np.ndarray:
    """Connected-component label of every vertex (smallest vertex id of its component)."""
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in zip(np.asarray(src).tolist(), np.asarray(dst).tolist()):
        ra, rb = find(a), find(b)
        if ra != rb:
            if ra < rb:
                parent[rb] = ra
            else:
                parent[ra] = rb
    return np.array([find(v) for v in range(n)], dtype=np.int64)


def int16_bound(n: int, src, dst, w):
    """Packed-16-bit enable test.

    For each connected component c with root r_c (its smallest vertex), the
    triangle inequality gives d(i,j) <= d(i,r_c) + d(r_c,j) <= 2 ecc(r_c) for
    every pair i, j in c.  Returns (bound, enabled) where bound is the maximum
    over components of 2 ecc(r_c) and enabled = bound < INF16.
    """
    lab = components(n, src, dst)
    roots = np.unique(lab)
    rows = dijkstra(n, src, dst, w, roots)
    bound = 0
    for r, row in zip(roots, rows):
        mine = row[lab == r]
        bound = max(bound, 2 * int(mine.max()))
    return bound, bound < INF16


def pack_u16(D32: np.ndarray) -> np.ndarray:
    """int32 distances -> unsigned 16-bit storage: INF32 -> INF16, finite d -> d.

    Defined only when every finite entry is < INF16 (the caller checks).
    """
    D32 = np.asarray(D32)
    out = D32.astype(np.int64)
    out[D32 >= INF32] = INF16
    if (out[D32 < INF32] >= INF16).any():
        raise ValueError("a finite distance does not fit below INF16")
    return out.astype(np.uint16)


def unpack_u16(D16: np.ndarray) -> np.ndarray:
    """unsigned 16-bit storage -> int32: INF16 -> INF32, d -> d."""
    D16 = np.asarray(D16).astype(np.int64)
    out = D16.copy()
    out[D16 >= INF16] = INF32
    return out.astype(np.int32)
