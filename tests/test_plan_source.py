"""The schedule model's round plan is the kernel's own (no GPU).

The all-rounds kernel and its host launcher share one planning function,
`solve_round` in `csrc/fw_kernels.cu` (with `sym_prefix`, `LaP2` and `TileMap`).
This test copies those definitions out of the sources unchanged, compiles them
for the host with g++, and checks, for many sizes, dtypes, modes and grids,
that they give the same plan as the Python model in `test_schedule_model.py`
(which drives the simulated runs), and that the plan keeps its own invariants.
"""
import os
import re
import shutil
import subprocess

import pytest

from tests import test_schedule_model as model

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1902_04446_gb300", "csrc")
FIELDS = ["p0", "p1", "R", "C", "row_x0", "col_y1", "n_prio", "n_p2row", "n_p2col", "n_fin", "b1", "b2", "b3",
          "len_t", "total"]


def _block(src, start_marker, with_template=True):
    """The definition that starts at start_marker (with its template line), up to its closing brace."""
    i = src.index(start_marker)
    if with_template:
        i = src.rindex("template", 0, i)
    j = src.index("{", i)
    depth = 0
    for k in range(j, len(src)):
        if src[k] == "{":
            depth += 1
        elif src[k] == "}":
            depth -= 1
            if depth == 0:
                end = k + 1
                if src[end:end + 1] == ";":
                    end += 1
                return src[i:end]
    raise AssertionError(f"unbalanced braces after {start_marker}")


@pytest.fixture(scope="module")
def plan_exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ needed")
    dev = open(os.path.join(CSRC, "fw_device.cuh")).read()
    ker = open(os.path.join(CSRC, "fw_kernels.cu")).read()
    parts = [
        _block(dev, "struct TileMap {"),
        _block(ker, "long long sym_prefix(", with_template=False),
        _block(ker, "struct LaP2 {"),
        re.search(r"constexpr int LA_TILE = .*?;\n", ker).group(0),
        re.search(r"constexpr int LA_FIN_ROWS = .*?;", ker).group(0),
        _block(ker, "struct SolveRound {", with_template=False),
        _block(ker, "inline SolveRound solve_round("),
    ]
    prog = "\n".join([
        "#include <cstdint>", "#include <cstdio>", "#include <cstdlib>",
        "#define __host__", "#define __device__", "#define __forceinline__ inline",
        "struct OpI32 { static constexpr int EPW = 1; };", "struct OpU16 { static constexpr int EPW = 2; };",
    ] + parts + ["""
template <class Op>
static void dump(int64_t n, int sym, int grid, bool has_rowP) {
  const int E = Op::EPW, q = (int)((n + 63) / 64);
  const int tiles_x = (int)((n + 128 * E - 1) / (128 * E)), tiles_y = (int)((n + 127) / 128);
  int tiles_total = 0;
  for (int y = 0; y < tiles_y; ++y) tiles_total += sym ? tiles_x - (y / E < tiles_x ? y / E : tiles_x) : tiles_x;
  if (grid > tiles_total) grid = tiles_total;
  for (int y = 0; y <= tiles_y; ++y) printf("S %d %lld\\n", y, sym_prefix(y, tiles_x, E));
  for (int j = 0; j <= q; ++j) {
    const SolveRound r = solve_round<Op, 64>(n, q, tiles_x, tiles_y, tiles_total, grid, sym, has_rowP, j);
    printf("R %d %lld %lld %d %d %d %d %d %d %d %d %d %d %d %d %d\\n", j, (long long)r.p0, (long long)r.p1, r.R,
           r.C, r.row_x0, r.col_y1, r.n_prio, r.n_p2row, r.n_p2col, r.n_fin, r.b1, r.b2, r.b3, r.len_t, r.total);
  }
}
int main(int argc, char **argv) {
  const int64_t n = atoll(argv[1]);
  const int epw = atoi(argv[2]), sym = atoi(argv[3]), grid = atoi(argv[4]), rowp = atoi(argv[5]);
  if (epw == 2) dump<OpU16>(n, sym, grid, rowp != 0);
  else dump<OpI32>(n, sym, grid, rowp != 0);
  return 0;
}
"""])
    d = tmp_path_factory.mktemp("plan")
    (d / "plan.cpp").write_text(prog)
    exe = d / "plan"
    subprocess.run(["g++", "-std=c++17", "-O1", "-o", str(exe), str(d / "plan.cpp")], check=True)
    return str(exe)


@pytest.mark.parametrize("n", [65, 130, 257, 1000, 2049, 4100, 8200, 16384, 24000])
@pytest.mark.parametrize("epw,sym", [(1, False), (1, True), (2, False), (2, True)])
@pytest.mark.parametrize("grid", [2, 152])
def test_source_plan_equals_model_and_keeps_its_invariants(plan_exe, n, epw, sym, grid):
    cfg = model.Cfg(n, epw, sym, grid_cap=grid)
    out = subprocess.run([plan_exe, str(n), str(epw), str(int(sym)), str(grid), str(int(cfg.has_rowP))],
                         capture_output=True, text=True, check=True).stdout.split("\n")
    sp = {int(a): int(b) for t, a, b in (l.split() for l in out if l.startswith("S "))}
    for y, v in sp.items():
        assert v == model.sym_prefix(y, cfg.tiles_x, epw) or not sym
    if sym:  # the prefix counts exactly the upper-band tiles of the rows above
        assert sp[cfg.tiles_y] == cfg.tiles_total
    rows = [list(map(int, l.split()[1:])) for l in out if l.startswith("R ")]
    assert len(rows) == cfg.q + 1
    block = 0
    for vals in rows:
        j, got = vals[0], dict(zip(FIELDS, vals[1:]))
        exp = cfg.round(j)
        for f in FIELDS:
            if f in ("row_x0", "col_y1", "R", "C") and j >= cfg.q:
                continue  # the last block has no tasks
            assert got[f] == exp[f], (j, f, got[f], exp[f])
        if 1 <= j < cfg.q:
            assert got["b1"] <= got["b2"] <= got["b3"] <= got["len_t"]
            assert got["total"] == got["len_t"] + 1 + got["n_p2row"] + got["n_p2col"] + got["n_fin"]
            assert got["len_t"] == got["n_prio"] + cfg.tiles_total
        if j >= 1:
            block = max(block, got["total"])
    assert block == cfg.block


@pytest.fixture(scope="module")
def decode_exe(tmp_path_factory):
    """The producer's item decode of the all-rounds kernel (its cached round, block and tile-row state
    included), copied out of the kernel's source unchanged and compiled for the host."""
    if shutil.which("g++") is None:
        pytest.skip("g++ needed")
    dev = open(os.path.join(CSRC, "fw_device.cuh")).read()
    ker = open(os.path.join(CSRC, "fw_kernels.cu")).read()
    a = ker.index("      SolveRound cr{};")
    b = ker.index("      // The producer never blocks on another item")
    chunk = ker[a:b]
    parts = [
        _block(dev, "struct TileMap {"),
        _block(ker, "long long sym_prefix(", with_template=False),
        _block(ker, "struct LaP2 {"),
        re.search(r"constexpr int LA_TILE = .*?;\n", ker).group(0),
        re.search(r"constexpr int LA_FIN_ROWS = .*?;", ker).group(0),
        _block(ker, "struct SolveRound {", with_template=False),
        _block(ker, "inline SolveRound solve_round("),
    ]
    prog = "\n".join([
        "#include <cstdint>", "#include <cstdio>", "#include <cstdlib>",
        "#define __host__", "#define __device__", "#define __forceinline__ inline",
        "struct OpI32 { static constexpr int EPW = 1; };", "struct OpU16 { static constexpr int EPW = 2; };",
    ] + parts + ["""
struct Plan { int q, tiles_x, tiles_y, tiles_total, grid, sym, block, base1; };
template <class Op>
static void run(int64_t n, int sym, int grid, bool has_rowP, long long start, int mode, unsigned seed, long long cap) {
  const int E = Op::EPW;
  Plan P{};
  P.q = (int)((n + 63) / 64);
  P.tiles_x = (int)((n + 128 * E - 1) / (128 * E));
  P.tiles_y = (int)((n + 127) / 128);
  for (int y = 0; y < P.tiles_y; ++y) P.tiles_total += sym ? P.tiles_x - (y / E < P.tiles_x ? y / E : P.tiles_x) : P.tiles_x;
  P.grid = grid < P.tiles_total ? grid : P.tiles_total;
  P.sym = sym;
  auto round_info = [&](int j) {
    return solve_round<Op, 64>(n, P.q, P.tiles_x, P.tiles_y, P.tiles_total, P.grid, P.sym, has_rowP, j);
  };
  P.base1 = round_info(0).total;
  for (int j = 1; j <= P.q; ++j) P.block = P.block > round_info(j).total ? P.block : round_info(j).total;
"""] + [chunk] + ["""
  const long long last = P.base1 + (long long)P.block * P.q + 1;
  unsigned s = seed;
  long long printed = 0;
  for (long long item = start; item <= last && printed < cap; ++printed) {
    int kind, rnd, info;
    decode(item, kind, rnd, info);
    printf("D %lld %d %d %d\\n", item, kind, rnd, info);
    long long step = 1;
    if (mode == 1) step = 152;
    if (mode == 2) {  // mostly short gaps, now and then a jump of up to two blocks
      s = s * 1664525u + 1013904223u;
      step = (s >> 28) == 0 ? 1 + (long long)((s >> 8) % (2 * (unsigned)P.block + 1)) : 1 + (long long)((s >> 8) % 300);
    }
    item += step;
  }
}
int main(int argc, char **argv) {
  const int64_t n = atoll(argv[1]);
  const int epw = atoi(argv[2]), sym = atoi(argv[3]), grid = atoi(argv[4]), rowp = atoi(argv[5]);
  const long long start = atoll(argv[6]);
  const int mode = atoi(argv[7]);
  const unsigned seed = (unsigned)atoi(argv[8]);
  const long long cap = atoll(argv[9]);
  if (epw == 2) run<OpU16>(n, sym, grid, rowp != 0, start, mode, seed, cap);
  else run<OpI32>(n, sym, grid, rowp != 0, start, mode, seed, cap);
  return 0;
}
"""])
    d = tmp_path_factory.mktemp("decode")
    (d / "decode.cpp").write_text(prog)
    exe = d / "decode"
    subprocess.run(["g++", "-std=c++17", "-O1", "-o", str(exe), str(d / "decode.cpp")], check=True)
    return str(exe)


@pytest.mark.parametrize("n,epw,sym", [(300, 1, True), (1000, 2, True), (2049, 1, False), (4100, 1, True),
                                       (4100, 2, True), (8200, 2, False), (24000, 1, True)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_kernel_item_decode_equals_model(decode_exe, n, epw, sym, mode):
    """Every item a CTA may take -- consecutive, every 152nd, or irregular increasing gaps with jumps across
    blocks -- decodes to the same kind, round and tile (or task index) as the model's plain decode: the kernel's
    cached round, block and tile-row state never changes an answer."""
    cfg = model.Cfg(n, epw, sym, grid_cap=152)
    cap = 60000
    out = subprocess.run([decode_exe, str(n), str(epw), str(int(sym)), "152", str(int(cfg.has_rowP)), "0",
                          str(mode), str(n + mode), str(cap)], capture_output=True, text=True, check=True).stdout
    seen = 0
    for line in out.split("\n"):
        if not line.startswith("D "):
            continue
        _, item, kind, rnd, info = line.split()
        item, kind, rnd, info = int(item), int(kind), int(rnd), int(info)
        ek, er, ei = cfg.decode(item)
        assert kind == ek, (item, kind, ek)
        if kind == model.TILE:
            assert rnd == er and ((info >> 16), info & 0xFFFF) == ei, (item, rnd, info, er, ei)
        elif kind in (model.P1, model.P2, model.FIN):
            assert rnd == er and (kind == model.P1 or info == ei), (item, kind, rnd, info, er, ei)
        elif kind == model.END:
            assert rnd == er
        seen += 1
    assert seen > 0
