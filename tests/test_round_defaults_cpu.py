"""The default round shape by n and element type, checked on the host (no GPU).

`default_phase3` and `default_round_width` in `csrc/fw_launch.h` choose, when
nothing was tuned, between one launch per round and every round in one launch,
and between 64- and 128-wide rounds.  This test copies both definitions out of
the header unchanged, compiles them with g++, and compares their table over n
and the three element types (0 int32, 1 packed 16-bit, 2 fp32) with the rule
the header documents, written out again here, and with the shapes that are
valid at all: every round in one launch only at width 64, width 128 only with
one launch per round.
"""
import os
import shutil
import subprocess

import pytest

from tests.test_plan_source import _block

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1902_04446_gb300", "csrc")

NS = [1, 127, 128, 2048, 4096, 5120, 6143, 6144, 8192, 16384, 24575, 24576, 32768, 49151, 49152, 65536, 262144]

MAIN = r"""
#include <cstdio>
#include <cstdlib>
int main(int argc, char **argv) {
  for (int i = 1; i < argc; ++i) {
    const long long n = atoll(argv[i]);
    for (int dt = 0; dt < 3; ++dt)
      printf("%lld %d %d %d\n", n, dt, apsp::default_phase3(n, dt), apsp::default_round_width(n, dt));
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ needed")
    hdr = open(os.path.join(CSRC, "fw_launch.h")).read()
    prog = "\n".join(["#include <cstdint>", "namespace apsp {",
                      _block(hdr, "inline int default_phase3(", with_template=False),
                      _block(hdr, "inline int default_round_width(", with_template=False), "}", MAIN])
    d = tmp_path_factory.mktemp("defaults")
    src, out = d / "defaults.cpp", d / "defaults"
    src.write_text(prog)
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", str(out), str(src)], check=True)
    res = subprocess.run([str(out)] + [str(n) for n in NS], check=True, capture_output=True, text=True).stdout
    return {(int(a), int(b)): (int(c), int(e)) for a, b, c, e in (line.split() for line in res.splitlines())}


def _rule(n, dt):
    """The documented defaults: every round in one launch (kernel 4) for 6144 <= n < 24576 (49152 for packed
    16-bit), one launch per round (kernel 3) otherwise; 128-wide rounds for packed 16-bit and fp32 where large n
    runs one launch per round, 64-wide otherwise."""
    hi = 49152 if dt == 1 else 24576
    p3 = 4 if 6144 <= n < hi else 3
    bk = 128 if dt != 0 and p3 == 3 and n >= 6144 else 64
    return p3, bk


@pytest.mark.parametrize("dt", [0, 1, 2])
def test_defaults_follow_the_documented_rule(table, dt):
    for n in NS:
        assert table[(n, dt)] == _rule(n, dt), (n, dt)


def test_default_shapes_are_valid_combinations(table):
    for (n, dt), (p3, bk) in table.items():
        assert bk in (64, 128) and p3 in (3, 4)
        assert not (p3 == 4 and bk != 64), (n, dt)  # the single launch is built for 64-wide rounds only


def test_int32_headline_shape_and_wide_rounds_at_large_n(table):
    assert table[(65536, 0)] == (3, 64)     # the n = 65536 int32 workload: one launch per round, width 64
    assert table[(65536, 1)] == (3, 128)    # its packed 16-bit line: width 128
    assert table[(262144, 1)] == (3, 128)
    assert table[(65536, 2)] == (3, 128)
    assert table[(16384, 2)] == (4, 64)     # fp32 at n = 16384: every round in one launch
    assert table[(4096, 1)] == (3, 64)      # small n: 64-wide rounds for every element type
