"""The upper-triangular storage layout, checked on the host (no GPU).

`Layout` and `tri_layout` in `csrc/fw_device.cuh` decide where every stored
element of the folded upper-triangular format lives.  This test copies both
definitions out of the source unchanged, compiles them with g++, and checks
for many n and both word widths that the map sends every stored element
(r, c) -- floor(c / S) >= floor(r / S), including the padding up to T S --
to a distinct position inside the rectangle, that the rectangle holds about
n^2 / 2 elements, and that the map agrees with the format's definition as
the header states it (written out again here in Python).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from tests.test_plan_source import _block

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1902_04446_gb300", "csrc")

MAIN = r"""
#include <cstdio>
#include <cstdlib>
int main(int argc, char **argv) {
  const long long n = atoll(argv[1]);
  const int epw = atoi(argv[2]);
  int64_t rows = 0;
  apsp::Layout L = apsp::tri_layout(n, epw, &rows);
  const long long S = 1ll << L.sh, end = (long long)L.T << L.sh;
  printf("%lld %lld %d %d %d %lld\n", (long long)rows, (long long)L.ld, L.sh, L.Th, L.T, end);
  for (long long r = 0; r < end; ++r)
    for (long long c = 0; c < end; ++c)
      if (L.stored(r, c)) printf("%lld\n", (long long)L.off(r, c));
  return 0;
}
"""


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ needed")
    dev = open(os.path.join(CSRC, "fw_device.cuh")).read()
    prog = "\n".join(["#include <cstdint>", "#define __host__", "#define __device__", "#define __forceinline__ inline",
                      "namespace apsp {", _block(dev, "struct Layout {", with_template=False),
                      _block(dev, "inline Layout tri_layout(", with_template=False), "}", MAIN])
    d = tmp_path_factory.mktemp("tri")
    src, out = d / "tri.cpp", d / "tri"
    src.write_text(prog)
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", str(out), str(src)], check=True)
    return str(out)


def _definition(n, epw):
    """The format as documented: S = 128 epw, T = ceil(n / S), Th = ceil(T / 2), pitch (2 Th + 1) S; super-row I
    < Th in rectangle rows I S.. shifted right by S, super-row I >= Th in rows (2 Th - 1 - I) S.. shifted left by I S."""
    S = 128 * epw
    T = -(-n // S)
    Th = -(-T // 2)
    ld = (2 * Th + 1) * S
    offs = []
    for r in range(T * S):
        I = r // S
        for c in range(I * S, T * S):
            pr, pc = (r, c + S) if I < Th else ((2 * Th - 1 - I) * S + (r - I * S), c - I * S)
            offs.append(pr * ld + pc)
    return Th * S, ld, np.array(offs, dtype=np.int64)


@pytest.mark.parametrize("n,epw", [(1, 1), (100, 1), (128, 1), (129, 1), (384, 1), (700, 1), (1000, 1), (1, 2),
                                   (256, 2), (257, 2), (600, 2), (1300, 2)])
def test_every_stored_element_has_its_own_place_in_the_rectangle(exe, n, epw):
    out = subprocess.run([exe, str(n), str(epw)], capture_output=True, text=True, check=True).stdout.split("\n")
    rows, ld, sh, Th, T, end = (int(x) for x in out[0].split())
    offs = np.array([int(x) for x in out[1:] if x], dtype=np.int64)
    S = 1 << sh
    assert S == 128 * epw and T == -(-n // S) and end == T * S
    assert offs.size == S * S * T * (T + 1) // 2  # the super-tiles (I, J) with I <= J
    assert offs.min() >= 0 and offs.max() < rows * ld  # inside the rectangle
    assert np.unique(offs).size == offs.size  # no two elements share a place
    r_rows, r_ld, r_offs = _definition(n, epw)
    assert (rows, ld) == (r_rows, r_ld)
    np.testing.assert_array_equal(offs, r_offs)
    if T >= 4:
        assert rows * ld <= 0.5 * (T * S) ** 2 * (1 + 3.0 / T)  # about half of the dense padded square
