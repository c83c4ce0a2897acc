"""Full-size workloads through apsp_solve_edges, against the oracle.

* roll64k: n = 65536 Swiss-roll kNN, solved in int32 and in packed 16-bit
  (auto bound); both matrices are compared element by element with the
  oracle's Dijkstra from every one of the 65536 sources (row chunks, threads),
  plus whole-matrix properties (zero diagonal, symmetry, no INF in a
  connected graph).
* roll256k: n = 262144 Swiss-roll kNN, packed 16-bit, solved in place twice:
  as a dense matrix (137 GB on the device) and in upper-triangular storage
  (68.8 GB), about four minutes each; 4096 seeded sample rows of each against
  the oracle's Dijkstra (a full oracle pass is out of reach at this size).
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _edges_dev(g, wdtype):
    return (torch.from_numpy(g.src.astype(np.int32)).cuda(), torch.from_numpy(g.dst.astype(np.int32)).cuda(),
            torch.from_numpy(g.w.astype(wdtype)).cuda())


def _as_i64(D_rows, u16):
    got = D_rows.cpu().numpy()
    if u16:
        got = oracle.unpack_u16(got.view(np.uint16))
    return got.astype(np.int64)


def _check_rows(D, g, rows, u16, chunk=512):
    for i in range(0, rows.shape[0], chunk):  # bounded host memory at n = 262144
        rs = rows[i:i + chunk]
        got = _as_i64(D[torch.from_numpy(rs).cuda().long()], u16)
        np.testing.assert_array_equal(got, oracle.dijkstra(g.n, g.src, g.dst, g.w, rs))


def _whole_matrix_properties(D, inf):
    n = D.shape[0]
    assert bool((torch.diagonal(D) == 0).all())
    assert not bool((D == inf).any())  # the graph is connected
    # symmetry, checked block by block to bound the temporary memory
    step = 8192
    for i in range(0, n, step):
        for j in range(i, n, step):
            assert torch.equal(D[i:i + step, j:j + step], D[j:j + step, i:i + step].T)


def test_roll64k_int32_and_packed16_whole_matrix(lib):
    """Both element types of the n = 65536 workload, every entry against the oracle (Dijkstra from all 65536
    sources, computed once and compared with both results)."""
    g = gen.workload("roll64k")
    bound, ok = oracle.int16_bound(g.n, g.src, g.dst, g.w)
    assert ok, bound
    with lib.Handle(device=0) as h:
        src, dst, w = _edges_dev(g, np.int32)
        D32 = h.solve_edges("int32", src, dst, w, g.n)
        assert h.last_status() == 0
        src, dst, w16 = _edges_dev(g, np.int16)
        D16 = h.solve_edges("u16", src, dst, w16, g.n)  # the bound is checked on the device first
        assert h.last_status() == 0
        _whole_matrix_properties(D32, lib.INF_I32)
        _whole_matrix_properties(D16, lib.INF_U16)
        chunk = 2048
        for r0 in range(0, g.n, chunk):
            rows = np.arange(r0, min(g.n, r0 + chunk))
            exp = oracle.dijkstra(g.n, g.src, g.dst, g.w, rows)
            np.testing.assert_array_equal(_as_i64(D32[r0:r0 + rows.shape[0]], False), exp)
            np.testing.assert_array_equal(_as_i64(D16[r0:r0 + rows.shape[0]], True), exp)
        del D32, D16
        torch.cuda.empty_cache()


def test_roll256k_packed16_in_place_sampled_rows(lib):
    g = gen.workload("roll256k")
    bound, ok = oracle.int16_bound(g.n, g.src, g.dst, g.w)
    assert ok, bound
    with lib.Handle(device=0) as h:
        src, dst, w = _edges_dev(g, np.int16)
        D = torch.empty((g.n, g.n), dtype=torch.int16, device="cuda")  # 137 GB, solved in place
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h.solve_edges("u16", src, dst, w, g.n, D)
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        print(f"\nroll256k packed-16 solve: {sec:.1f} s, {g.n ** 3 / sec / 1e12:.2f} TRelax/s (bound {bound})")
        assert h.last_status() == 0
        rng = np.random.default_rng(262144)
        _check_rows(D, g, np.sort(rng.choice(g.n, size=4096, replace=False)), u16=True)
        assert bool((torch.diagonal(D) == 0).all())
        del D
        torch.cuda.empty_cache()


def test_roll256k_packed16_upper_triangular_storage_sampled_rows(lib):
    """The n = 262144 workload in half the memory: the edge list into upper-triangular storage (68.8 GB instead of
    137 GB), solved in place; 4096 sampled rows, read back by apsp_tri_rows, equal the oracle's Dijkstra rows."""
    g = gen.workload("roll256k")
    rows_, ld, nbytes = lib.tri_layout("u16", g.n)
    assert nbytes < 0.51 * g.n * g.n * 2
    with lib.Handle(device=0) as h:
        src, dst, w = _edges_dev(g, np.int16)
        T = h.tri_from_edges("u16", src, dst, w, g.n)  # the 16-bit bound is checked first
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h.solve_tri("u16", T, g.n)
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        print(f"\nroll256k packed-16 upper-triangular solve: {sec:.1f} s, {g.n ** 3 / sec / 1e12:.2f} TRelax/s, "
              f"{nbytes / 1e9:.1f} GB")
        assert h.last_status() == 0
        rng = np.random.default_rng(262145)
        rows = np.sort(rng.choice(g.n, size=4096, replace=False))
        for i in range(0, rows.shape[0], 512):
            rs = rows[i:i + 512]
            got = lib.tri_rows("u16", T, g.n, torch.from_numpy(rs).cuda())
            np.testing.assert_array_equal(_as_i64(got, True), oracle.dijkstra(g.n, g.src, g.dst, g.w, rs))
        del T
        torch.cuda.empty_cache()
