"""The oracle's pins catch plausible mistakes.

Each test copies ``oracle/apsp_oracle.c`` to a temporary directory, plants one
mistake in the copy (a dropped term, a wrong index, a transposed operand, an
off-by-one, a flipped comparison, a wrong heap order), compiles it, and checks
that the pin guarding that routine no longer agrees; the same harness on an
unchanged copy agrees with every pin.  The committed oracle is never modified.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from tests import pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "apsp_oracle.c")

MUTANTS = {
    "dropped_term": ("int64_t via = dik + dkj;", "int64_t via = dkj;"),
    "transposed_operand": ("int64_t dkj = d[k * n + j];", "int64_t dkj = d[j * n + k];"),
    "wrong_row_index": ("int64_t dik = d[i * n + k];", "int64_t dik = d[k * n + i];"),
    "off_by_one_k": ("for (int64_t k = k_begin; k < k_end; ++k) {\n    for (int64_t i = 0; i < n; ++i) {\n      int64_t dik",
                     "for (int64_t k = k_begin; k < k_end - 1; ++k) {\n    for (int64_t i = 0; i < n; ++i) {\n      int64_t dik"),
    "flipped_compare": ("if (via < d[i * n + j]) d[i * n + j] = via;", "if (via > d[i * n + j]) d[i * n + j] = via;"),
    # the classic loop-order mistake: k innermost instead of outermost
    "k_innermost": None,
}


K_INNERMOST = """int oracle_fw_i64(int64_t *d, int64_t n, int64_t inf, int64_t k_begin, int64_t k_end) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j)
      for (int64_t k = k_begin; k < k_end; ++k) {
        if (d[i * n + k] == inf || d[k * n + j] == inf) continue;
        if (d[i * n + k] + d[k * n + j] < d[i * n + j]) d[i * n + j] = d[i * n + k] + d[k * n + j];
      }
  return 0;
}

"""


def _compile(tmp_path, name, old, new):
    src = open(SRC).read()
    if old is None:
        a = src.index("int oracle_fw_i64(")
        b = src.index("/* Same in double precision")
        mut = src[:a] + K_INNERMOST + src[b:]
    else:
        assert src.count(old) >= 1, f"mutation anchor for {name} not found"
        mut = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(mut)
    subprocess.run(["gcc", "-O1", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-shared", "-fPIC", "-pthread",
                    "-o", str(so), str(c), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_fw_i64.argtypes = [i64p] + [ctypes.c_int64] * 4
    lib.oracle_fw_i64.restype = ctypes.c_int
    return lib


def _run(lib, W):
    d = np.ascontiguousarray(W, dtype=np.int64).copy()
    n = d.shape[0]
    lib.oracle_fw_i64(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n, pins.INF, 0, n)
    return d


def _fw_i64_caught(lib):
    for seed in range(20):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(3, 9))
        directed = seed % 2 == 1
        edges = pins.random_graph(rng, n, 0.45, wmax=20, directed=directed)
        W = pins.dense(n, edges, directed)
        if not np.array_equal(_run(lib, W), pins.brute_force(n, edges, directed)):
            return True
    return False


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc needed")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_brute_force_pin_catches_mutant(tmp_path, name):
    old, new = MUTANTS[name] or (None, None)
    lib = _compile(tmp_path, name, old, new)
    assert _fw_i64_caught(lib), f"mutant {name} survived the brute-force pin"


# Mistakes planted in the oracle's other routines, each against the pin that
# guards it: the min-plus product against its loop definition, Dijkstra and
# the float Floyd-Warshall against brute-force path enumeration.
OTHER_MUTANTS = {
    "minplus_drops_C": ("minplus", "int64_t best = C[i * nn + j];", "int64_t best = inf;"),
    "minplus_skips_last_t": ("minplus", "for (int64_t t = 0; t < kk; ++t) {\n        int64_t a = A[i * kk + t]",
                             "for (int64_t t = 0; t + 1 < kk; ++t) {\n        int64_t a = A[i * kk + t]"),
    "minplus_wrong_B_index": ("minplus", "int64_t a = A[i * kk + t], b = B[t * nn + j];",
                              "int64_t a = A[i * kk + t], b = B[(j % kk) * nn + (t % nn)];"),
    "dijkstra_unit_weights": ("dijkstra", "int64_t nd = u.ikey + J->wi[e];", "int64_t nd = u.ikey + 1;"),
    "dijkstra_max_heap": ("dijkstra", "return h->use_double ? (x->key < y->key) : (x->ikey < y->ikey);",
                          "return h->use_double ? (x->key < y->key) : (x->ikey > y->ikey);"),
    "dijkstra_skips_first_edge": ("dijkstra", "for (int64_t e = J->rowptr[u.v]; e < J->rowptr[u.v + 1]; ++e) {",
                                  "for (int64_t e = J->rowptr[u.v] + 1; e < J->rowptr[u.v + 1]; ++e) {"),
    "fw_f64_dropped_term": ("fw_f64", "double via = dik + dkj;", "double via = dkj;"),
}


def _minplus_caught(lib):
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_minplus_i64.argtypes = [i64p, i64p, i64p] + [ctypes.c_int64] * 4
    lib.oracle_minplus_i64.restype = ctypes.c_int
    for seed in range(10):
        rng = np.random.default_rng(100 + seed)
        m, kk, nn = (int(x) for x in rng.integers(2, 9, size=3))
        A = rng.integers(0, 50, size=(m, kk)).astype(np.int64)
        B = rng.integers(0, 50, size=(kk, nn)).astype(np.int64)
        C = rng.integers(0, 120, size=(m, nn)).astype(np.int64)
        A[rng.random(A.shape) < 0.3] = pins.INF
        B[rng.random(B.shape) < 0.3] = pins.INF
        got = C.copy()
        lib.oracle_minplus_i64(A.ctypes.data_as(i64p), B.ctypes.data_as(i64p), got.ctypes.data_as(i64p),
                               m, kk, nn, pins.INF)
        exp = C.copy()
        for i in range(m):
            for j in range(nn):
                for t in range(kk):
                    if A[i, t] < pins.INF and B[t, j] < pins.INF:
                        exp[i, j] = min(exp[i, j], A[i, t] + B[t, j])
        if not np.array_equal(got, exp):
            return True
    return False


def _dijkstra_caught(lib):
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_dijkstra_i64.argtypes = [ctypes.c_int64, i64p, i64p, i64p, i64p, ctypes.c_int64, i64p,
                                        ctypes.c_int64, ctypes.c_int]
    lib.oracle_dijkstra_i64.restype = ctypes.c_int
    for seed in range(20):
        rng = np.random.default_rng(200 + seed)
        n = int(rng.integers(3, 9))
        directed = seed % 2 == 1
        edges = pins.random_graph(rng, n, 0.45, wmax=20, directed=directed)
        if not edges:
            continue
        s = np.array([e[0] for e in edges]); d = np.array([e[1] for e in edges]); w = np.array([e[2] for e in edges])
        if not directed:
            s, d, w = np.concatenate([s, d]), np.concatenate([d, s]), np.concatenate([w, w])
        order = np.argsort(s, kind="stable")
        col = np.ascontiguousarray(d[order], dtype=np.int64)
        ww = np.ascontiguousarray(w[order], dtype=np.int64)
        rowptr = np.zeros(n + 1, dtype=np.int64)
        np.add.at(rowptr, s + 1, 1)
        rowptr = np.ascontiguousarray(np.cumsum(rowptr), dtype=np.int64)
        src = np.arange(n, dtype=np.int64)
        out = np.empty((n, n), dtype=np.int64)
        lib.oracle_dijkstra_i64(n, rowptr.ctypes.data_as(i64p), col.ctypes.data_as(i64p), ww.ctypes.data_as(i64p),
                                src.ctypes.data_as(i64p), n, out.ctypes.data_as(i64p), pins.INF, 1)
        if not np.array_equal(out, pins.brute_force(n, edges, directed)):
            return True
    return False


def _fw_f64_caught(lib):
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.oracle_fw_f64.argtypes = [f64p] + [ctypes.c_int64] * 3
    lib.oracle_fw_f64.restype = ctypes.c_int
    for seed in range(20):
        rng = np.random.default_rng(300 + seed)
        n = int(rng.integers(3, 9))
        edges = pins.random_graph(rng, n, 0.45, wmax=20)
        exp = pins.brute_force(n, edges).astype(np.float64) / 4.0  # quarter weights: exact in binary
        exp[exp >= pins.INF / 4.0] = np.inf
        W = np.full((n, n), np.inf)
        np.fill_diagonal(W, 0.0)
        for u, v, w in edges:
            W[u, v] = W[v, u] = min(W[u, v], w / 4.0)
        lib.oracle_fw_f64(W.ctypes.data_as(f64p), n, 0, n)
        if not np.array_equal(W, exp):
            return True
    return False


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc needed")
@pytest.mark.parametrize("name", sorted(OTHER_MUTANTS))
def test_pins_catch_mutants_in_other_routines(tmp_path, name):
    family, old, new = OTHER_MUTANTS[name]
    lib = _compile(tmp_path, name, old, new)
    caught = {"minplus": _minplus_caught, "dijkstra": _dijkstra_caught, "fw_f64": _fw_f64_caught}[family](lib)
    assert caught, f"mutant {name} survived its pin"


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc needed")
def test_unmutated_copy_passes_every_pin(tmp_path):
    """The same harness on the committed oracle, unchanged, finds nothing (the pins are not trivially failing)."""
    lib = _compile(tmp_path, "clean", "int oracle_fw_i64(", "int oracle_fw_i64(")
    assert not _fw_i64_caught(lib)
    assert not _minplus_caught(lib) and not _dijkstra_caught(lib) and not _fw_f64_caught(lib)


# Mistakes planted in a copy of the oracle's Python routines (the module's
# source with one line changed, executed in a fresh namespace; it loads the
# same committed C library).
ORACLE_PY = os.path.join(os.path.dirname(SRC), "__init__.py")
PY_MUTANTS = {
    "components_no_union": ("                parent[rb] = ra", "                parent[rb] = rb"),
    "bound_without_factor_2": ("bound = max(bound, 2 * int(mine.max()))", "bound = max(bound, int(mine.max()))"),
    "bound_over_whole_row": ("mine = row[lab == r]", "mine = row"),
}


def _py_mutant(name):
    import types
    old, new = PY_MUTANTS[name]
    src = open(ORACLE_PY).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found"
    ns = {"__file__": ORACLE_PY, "__name__": f"oracle_{name}"}
    exec(compile(src.replace(old, new), ORACLE_PY, "exec"), ns)
    return types.SimpleNamespace(**ns)


def _py_pins_fail(o):
    """The CPU pins of components and int16_bound, run against module o; True when one of them fails."""
    # components: INF exactly across components, against brute force on small graphs
    for seed in range(10):
        rng = np.random.default_rng(400 + seed)
        n = int(rng.integers(3, 9))
        edges = pins.random_graph(rng, n, 0.3, wmax=9)
        s = np.array([e[0] for e in edges], dtype=np.int64); d = np.array([e[1] for e in edges], dtype=np.int64)
        lab = o.components(n, s, d)
        same = lab[:, None] == lab[None, :]
        if not np.array_equal(same, pins.brute_force(n, edges) < pins.INF):
            return True
    # int16_bound: closed forms on a path and on two disjoint paths
    s = np.arange(39); d = s + 1
    if o.int16_bound(40, s, d, np.full(39, 9)) != (2 * 39 * 9, True):
        return True
    s = np.array([0, 1, 2, 3, 5, 6, 7]); d = s + 1
    if o.int16_bound(9, s, d, np.array([3, 3, 3, 3, 7, 7, 7])) != (42, True):
        return True
    return False


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_pins_catch_mutants_in_python_routines(name):
    assert _py_pins_fail(_py_mutant(name)), f"mutant {name} survived its pin"


def test_python_pins_pass_on_the_oracle():
    import oracle
    assert not _py_pins_fail(oracle)
