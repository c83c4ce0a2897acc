"""The oracle's pins catch plausible mistakes.

Each test copies ``oracle/apsp_oracle.c`` to a temporary directory, plants one
mistake in the copy (a dropped term, a wrong index, a transposed operand, an
off-by-one, a flipped comparison), compiles it, and checks that the brute-force
pin no longer agrees.  The committed oracle is never modified.
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


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc needed")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_brute_force_pin_catches_mutant(tmp_path, name):
    old, new = MUTANTS[name] or (None, None)
    lib = _compile(tmp_path, name, old, new)
    caught = False
    for seed in range(20):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(3, 9))
        directed = seed % 2 == 1
        edges = pins.random_graph(rng, n, 0.45, wmax=20, directed=directed)
        W = pins.dense(n, edges, directed)
        if not np.array_equal(_run(lib, W), pins.brute_force(n, edges, directed)):
            caught = True
            break
    assert caught, f"mutant {name} survived the brute-force pin"
