"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Integer results must be bit-exact.  fp32 results must be within 1e-4
relative of the float64 oracle, with exactly the same set of +inf entries.
Inputs come from the seeded generators in ``gen``; expected values only from
``oracle``.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
INF = oracle.INF32
REL_TOL = 1e-4   # fp32 vs float64 oracle: |d - d64| <= 1e-4 d64


@pytest.fixture(scope="module")
def H(lib):
    h = lib.Handle(device=0)
    yield h
    h.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def er_edges(n, seed, deg=4.0, wmax=100, directed=False):
    rng = np.random.default_rng(seed)
    m = int(deg * n / (1 if directed else 2))
    s = rng.integers(0, n, size=m)
    d = rng.integers(0, n, size=m)
    keep = s != d
    s, d = s[keep], d[keep]
    w = rng.integers(1, wmax + 1, size=s.shape[0])
    return s, d, w


def dense_directed(n, s, d, w, ld=None, dtype=np.int32, inf=INF):
    return gen.dense_matrix(n, s, d, w, dtype=dtype, inf=inf, ld=ld, directed=True)


def expect_fw(W):
    return oracle.fw(np.asarray(W)[:, : W.shape[0]].astype(np.int64))


# ------------------------------------------------------------------ min-plus product
@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (7, 3, 5), (128, 64, 128), (130, 65, 257), (300, 200, 140)])
@pytest.mark.parametrize("dt", ["int32", "u16", "fp32"])
def test_minplus_matches_oracle(H, m, k, n, dt):
    rng = np.random.default_rng(m * 1000 + k * 10 + n)
    if dt == "fp32":
        A = rng.random((m, k), dtype=np.float32) * 50
        B = rng.random((k, n), dtype=np.float32) * 50
        C = rng.random((m, n), dtype=np.float32) * 120
        A[rng.random(A.shape) < 0.2] = np.inf
        B[rng.random(B.shape) < 0.2] = np.inf
        got = H.minplus(dev(A), dev(B), dev(C)).cpu().numpy().astype(np.float64)
        exp = oracle.minplus(A.astype(np.float64), B.astype(np.float64), C.astype(np.float64))
        np.testing.assert_array_equal(np.isinf(got), np.isinf(exp))
        f = np.isfinite(exp)
        np.testing.assert_allclose(got[f], exp[f], rtol=REL_TOL, atol=0)
        return
    inf = INF if dt == "int32" else 0x7FFF
    hi = 5000 if dt == "int32" else 16000
    npdt = np.int32 if dt == "int32" else np.int16
    A = rng.integers(0, hi, size=(m, k)); B = rng.integers(0, hi, size=(k, n)); C = rng.integers(0, 2 * hi, size=(m, n))
    A[rng.random(A.shape) < 0.2] = inf
    B[rng.random(B.shape) < 0.2] = inf
    C[rng.random(C.shape) < 0.2] = inf
    got = H.minplus(dev(A.astype(npdt)), dev(B.astype(npdt)), dev(C.astype(npdt))).cpu().numpy().astype(np.int64)
    A64, B64, C64 = (np.where(x == inf, INF, x).astype(np.int64) for x in (A, B, C))
    exp = oracle.minplus(A64, B64, C64)
    if dt == "u16":
        exp = np.where(exp >= 0x7FFF, 0x7FFF, exp)   # INF16 (and sums >= INF16 never win over C <= INF16)
    np.testing.assert_array_equal(got, exp)


def _minplus_inputs(rng, m, k, n, dt):
    """A, B, C of the given dtype (INF entries included) and the oracle's C = min(C, A (x) B)."""
    if dt == "fp32":
        A = rng.random((m, k), dtype=np.float32) * 50
        B = rng.random((k, n), dtype=np.float32) * 50
        C = rng.random((m, n), dtype=np.float32) * 120
        A[rng.random(A.shape) < 0.2] = np.inf
        B[rng.random(B.shape) < 0.2] = np.inf
        return A, B, C, oracle.minplus(A.astype(np.float64), B.astype(np.float64), C.astype(np.float64))
    inf = INF if dt == "int32" else 0x7FFF
    hi = 5000 if dt == "int32" else 16000
    npdt = np.int32 if dt == "int32" else np.int16
    A = rng.integers(0, hi, size=(m, k)); B = rng.integers(0, hi, size=(k, n)); C = rng.integers(0, 2 * hi, size=(m, n))
    A[rng.random(A.shape) < 0.2] = inf
    B[rng.random(B.shape) < 0.2] = inf
    C[rng.random(C.shape) < 0.2] = inf
    A64, B64, C64 = (np.where(x == inf, INF, x).astype(np.int64) for x in (A, B, C))
    exp = oracle.minplus(A64, B64, C64)
    if dt == "u16":
        exp = np.where(exp >= 0x7FFF, 0x7FFF, exp)
    return A.astype(npdt), B.astype(npdt), C.astype(npdt), exp


@pytest.mark.parametrize("m,k,n", [(128, 64, 128), (333, 130, 261), (129, 64, 5), (70, 700, 300),
                                   (1024, 1024, 1024)])
@pytest.mark.parametrize("dt", ["int32", "u16", "fp32"])
def test_minplus_tma_path_padded_ld(H, m, k, n, dt):
    """B and C 16-byte addressable (leading dimensions padded to 8 elements): the TMA-fed product, with k in
    several 64-wide chunks, ragged m, n not a multiple of 4 (the columns after the last 16-byte unit are merged
    outside the int32 TMA reduction), and the padding columns of C left untouched."""
    rng = np.random.default_rng(m * 7 + k * 3 + n)
    A, B, C, exp = _minplus_inputs(rng, m, k, n, dt)
    pad = lambda x: (x + 7) // 8 * 8
    sentinel = 7
    bufs = []
    for X in (A, B, C):
        P = np.full((X.shape[0], pad(X.shape[1])), sentinel, dtype=X.dtype)
        P[:, :X.shape[1]] = X
        bufs.append(dev(P))
    Av, Bv, Cv = bufs[0][:, :k], bufs[1][:, :n], bufs[2][:, :n]
    H.minplus(Av, Bv, Cv)
    assert H.last_status() == 0
    out = bufs[2].cpu().numpy()
    assert (out[:, n:] == sentinel).all()
    got = out[:, :n]
    if dt == "fp32":
        got = got.astype(np.float64)
        np.testing.assert_array_equal(np.isinf(got), np.isinf(exp))
        f = np.isfinite(exp)
        np.testing.assert_allclose(got[f], exp[f], rtol=REL_TOL, atol=0)
    else:
        np.testing.assert_array_equal(got.astype(np.int64), exp)


# ------------------------------------------------------------------ repeated squaring (Alg. 1)
@pytest.mark.parametrize("n", [1, 2, 3, 65, 129, 300])
@pytest.mark.parametrize("dt", ["int32", "u16", "fp32"])
def test_squaring_solver_matches_oracle(H, n, dt):
    s, d, w = er_edges(n, seed=n + 5, deg=3.0, wmax=40)
    E = expect_fw(gen.dense_matrix(n, s, d, w, dtype=np.int32))
    if dt == "int32":
        D = H.solve_squaring(dt, dev(gen.dense_matrix(n, s, d, w, dtype=np.int32))).cpu().numpy().astype(np.int64)
    elif dt == "u16":
        D16 = H.solve_squaring(dt, dev(gen.dense_matrix(n, s, d, w, dtype=np.int16, inf=0x7FFF))).cpu().numpy()
        D = oracle.unpack_u16(D16.view(np.uint16)).astype(np.int64)
    else:
        Df = H.solve_squaring(dt, dev(gen.dense_matrix(n, s, d, w, dtype=np.float32))).cpu().numpy()
        D = np.where(np.isinf(Df), INF, Df.astype(np.float64)).astype(np.int64)  # small integers: exact
    assert H.last_status() == 0
    np.testing.assert_array_equal(D, E)


@pytest.mark.parametrize("n,ld", [(130, 136), (200, 201)])
def test_squaring_solver_directed_and_ld(H, n, ld):
    """Directed input; a 16-byte addressable ld (TMA-fed product) and an odd one (the kernel without workspace)."""
    s, d, w = er_edges(n, seed=ld, deg=3.0, wmax=90, directed=True)
    W = dense_directed(n, s, d, w, ld=ld)
    D = H.solve_squaring("int32", dev(W)).cpu().numpy()[:, :n]
    assert H.last_status() == 0
    np.testing.assert_array_equal(D.astype(np.int64), expect_fw(W))


# ------------------------------------------------------------------ int32 solves, odd sizes
@pytest.mark.parametrize("n", [1, 2, 3, 31, 33, 63, 64, 65, 127, 129, 200, 257, 513, 1000])
def test_int32_solve_odd_sizes_bit_exact(H, n):
    s, d, w = er_edges(n, seed=n, deg=3.0, wmax=1000)
    W = gen.dense_matrix(n, s, d, w, dtype=np.int32)
    D = H.solve_t("int32", dev(W)).cpu().numpy()
    assert H.last_status() == 0
    np.testing.assert_array_equal(D.astype(np.int64), expect_fw(W))


@pytest.mark.parametrize("n,ld", [(100, 103), (129, 136), (250, 257)])
def test_int32_padded_and_unaligned_leading_dimension(H, n, ld):
    s, d, w = er_edges(n, seed=ld, deg=3.0)
    W = gen.dense_matrix(n, s, d, w, dtype=np.int32, ld=ld)
    Wd = dev(W)
    guard = Wd[:, n:].clone()
    D = H.solve_t("int32", Wd)
    np.testing.assert_array_equal(D[:, :n].cpu().numpy().astype(np.int64), expect_fw(W))
    # in place: the padding columns beyond n are never written
    H.solve_t("int32", Wd, Wd)
    np.testing.assert_array_equal(Wd[:, :n].cpu().numpy().astype(np.int64), expect_fw(W))
    assert torch.equal(Wd[:, n:], guard)


@pytest.mark.parametrize("n", [70, 300, 777])
def test_directed_input_solved_exactly(H, n):
    """Directed graphs: the row and column panels use both operand orders."""
    s, d, w = er_edges(n, seed=n + 7, deg=4.0, directed=True)
    W = dense_directed(n, s, d, w)
    D = H.solve_t("int32", dev(W)).cpu().numpy()
    np.testing.assert_array_equal(D.astype(np.int64), expect_fw(W))


def test_disconnected_pairs_stay_exactly_inf(H):
    n = 400
    s, d, w = er_edges(n, seed=3, deg=0.7, wmax=1000)
    W = gen.dense_matrix(n, s, d, w, dtype=np.int32)
    D = H.solve_t("int32", dev(W)).cpu().numpy().astype(np.int64)
    E = expect_fw(W)
    assert (E == INF).any()
    np.testing.assert_array_equal(D, E)
    lab = oracle.components(n, s, d)
    assert ((D == INF) == (lab[:, None] != lab[None, :])).all()


def test_swiss_roll_512_int32(H):
    g = gen.workload("roll512")
    W = gen.dense_matrix(g.n, g.src, g.dst, g.w, dtype=np.int32)
    D = H.solve_t("int32", dev(W)).cpu().numpy()
    np.testing.assert_array_equal(D.astype(np.int64), expect_fw(W))


def test_large_weights_near_inf_do_not_overflow(H):
    n = 130
    s = np.arange(n - 1); d = s + 1
    w = np.full(n - 1, (INF - 1) // (n - 1))
    W = gen.dense_matrix(n, s, d, w, dtype=np.int32)
    D = H.solve_t("int32", dev(W)).cpu().numpy()
    np.testing.assert_array_equal(D.astype(np.int64), expect_fw(W))


# ------------------------------------------------------------------ packed 16-bit
@pytest.mark.parametrize("n", [5, 64, 100, 257, 600])
def test_u16_solve_bit_exact(H, n):
    s, d, w = er_edges(n, seed=n + 1, deg=3.0, wmax=60)
    W16 = gen.dense_matrix(n, s, d, w, dtype=np.int16, inf=0x7FFF)
    D16 = H.solve_t("u16", dev(W16)).cpu().numpy()
    E = expect_fw(gen.dense_matrix(n, s, d, w, dtype=np.int32))
    assert E[E < INF].max() < 0x7FFF
    np.testing.assert_array_equal(oracle.unpack_u16(D16.view(np.uint16)).astype(np.int64), E)


def test_u16_odd_leading_dimension(H):
    n, ld = 201, 203
    s, d, w = er_edges(n, seed=11, deg=3.0, wmax=60)
    W16 = gen.dense_matrix(n, s, d, w, dtype=np.int16, inf=0x7FFF, ld=ld)
    D16 = H.solve_t("u16", dev(W16)).cpu().numpy()[:, :n]
    E = expect_fw(gen.dense_matrix(n, s, d, w, dtype=np.int32))
    np.testing.assert_array_equal(oracle.unpack_u16(D16.view(np.uint16)).astype(np.int64), E)


def test_auto_uses_bound_and_matches_oracle(H):
    g = gen.workload("roll512")
    W = gen.dense_matrix(g.n, g.src, g.dst, g.w, dtype=np.int32)
    bound, ok = H.int16_bound(dev(W))
    eb, eok = oracle.int16_bound(g.n, g.src, g.dst, g.w)
    assert (bound, ok) == (eb, eok) and ok
    D = H.solve_t("auto", dev(W)).cpu().numpy()
    np.testing.assert_array_equal(D.astype(np.int64), expect_fw(W))


def test_auto_falls_back_to_int32_when_bound_fails(H):
    n = 300
    s = np.arange(n - 1); d = s + 1
    w = np.full(n - 1, 200)   # path: 2 ecc(0) = 2 * 299 * 200 > 32767
    W = gen.dense_matrix(n, s, d, w, dtype=np.int32)
    bound, ok = H.int16_bound(dev(W))
    assert bound == 2 * 299 * 200 and not ok
    D = H.solve_t("auto", dev(W)).cpu().numpy()
    np.testing.assert_array_equal(D.astype(np.int64), expect_fw(W))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_int16_bound_matches_oracle_disconnected(H, seed):
    n = 500
    s, d, w = er_edges(n, seed=seed + 40, deg=1.2, wmax=300)
    W = gen.dense_matrix(n, s, d, w, dtype=np.int32)
    assert H.int16_bound(dev(W)) == oracle.int16_bound(n, s, d, w)


def test_int16_bound_rejects_asymmetric(H):
    n = 50
    s, d, w = er_edges(n, seed=5, deg=3.0, directed=True)
    W = dense_directed(n, s, d, w)
    if (W == W.T).all():
        pytest.skip("generator produced a symmetric matrix")
    _, ok = H.int16_bound(dev(W))
    assert not ok


# ------------------------------------------------------------------ fp32
@pytest.mark.parametrize("n", [65, 300, 1000])
def test_fp32_within_tolerance(H, n):
    pts = gen.gaussian_mixture(n, seed=n, dim=10, components=3)
    s, d, dist = gen.knn_edges(pts, 6)
    w32 = dist.astype(np.float32)
    W = gen.dense_matrix(n, s, d, w32, dtype=np.float32)
    D = H.solve_t("fp32", dev(W)).cpu().numpy().astype(np.float64)
    E = oracle.fw(gen.dense_matrix(n, s, d, w32.astype(np.float64), dtype=np.float64))
    np.testing.assert_array_equal(np.isinf(D), np.isinf(E))
    f = np.isfinite(E) & (E > 0)
    assert (np.abs(D[f] - E[f]) <= REL_TOL * E[f]).all()
    assert (np.diag(D) == 0).all()


# ------------------------------------------------------------------ edge-list path
@pytest.mark.parametrize("dt", ["int32", "u16", "auto", "fp32"])
def test_solve_edges(H, dt):
    n = 333
    s, d, w = er_edges(n, seed=9, deg=3.0, wmax=50)
    # duplicates with larger weights and a self loop must not matter
    s2 = np.concatenate([s, s[:10], [4]]); d2 = np.concatenate([d, d[:10], [4]]); w2 = np.concatenate([w, w[:10] + 5, [1]])
    E = expect_fw(gen.dense_matrix(n, s, d, w, dtype=np.int32))
    wt = {"int32": np.int32, "auto": np.int32, "u16": np.int16, "fp32": np.float32}[dt]
    D = H.solve_edges(dt, dev(s2.astype(np.int32)), dev(d2.astype(np.int32)), dev(w2.astype(wt)), n).cpu().numpy()
    assert H.last_status() == 0
    if dt == "u16":
        D = oracle.unpack_u16(D.view(np.uint16))
    if dt == "fp32":
        D = np.where(np.isinf(D), INF, D.astype(np.float64))
    np.testing.assert_array_equal(D.astype(np.int64), E)


def test_solve_edges_u16_refuses_when_bound_fails(H, lib):
    n = 300
    s = np.arange(n - 1); d = s + 1
    w = np.full(n - 1, 200)
    with pytest.raises(lib.ApspError) as ei:
        H.solve_edges("u16", dev(s.astype(np.int32)), dev(d.astype(np.int32)), dev(w.astype(np.int16)), n)
    assert ei.value.name == "APSP_E_RANGE"


# ------------------------------------------------------------------ input checks
def test_input_checks_reported(H, lib):
    n = 40
    s, d, w = er_edges(n, seed=1)
    W = gen.dense_matrix(n, s, d, w, dtype=np.int32)
    bad = W.copy(); bad[3, 5] = -2
    H.solve_t("int32", dev(bad)); assert H.last_status() == 1
    bad = W.copy(); bad[7, 7] = 3
    H.solve_t("int32", dev(bad)); assert H.last_status() == 1
    bad = W.copy(); bad[1, 2] = INF + 5
    H.solve_t("int32", dev(bad)); assert H.last_status() == 4
    H.solve_t("int32", dev(W)); assert H.last_status() == 0
    with pytest.raises(ValueError):
        H.solve_t("int32", dev(W[:, :30]))   # the binding refuses a matrix narrower than n
    Wd = dev(W)
    # the C ABI itself refuses ld < n and null pointers before touching the device
    assert lib.lib.apsp_solve_t(H._h, 0, Wd.data_ptr(), n, n - 1, Wd.data_ptr(), None) == 1
    assert lib.lib.apsp_solve_t(H._h, 0, None, n, n, Wd.data_ptr(), None) == 1
    assert lib.lib.apsp_solve_t(H._h, 7, Wd.data_ptr(), n, n, Wd.data_ptr(), None) == 1
    Z = torch.zeros((0, 0), dtype=torch.int32, device="cuda")
    H.solve_t("int32", Z)


# ------------------------------------------------------------------ full-size workloads (sampled rows)
def _whole_matrix_check(D_dev, g, fp=False, chunk=2048):
    """Every row of the solved matrix against the oracle's Dijkstra from that source (row chunks bound the host
    memory): bit-exact for integer weights; for fp32 weights the +inf set is identical and every finite entry is
    within REL_TOL of the float64 distance."""
    n = g.n
    w = g.w.astype(np.float32).astype(np.float64) if fp else g.w
    for r0 in range(0, n, chunk):
        rows = np.arange(r0, min(n, r0 + chunk))
        got = D_dev[r0:r0 + rows.shape[0]].cpu().numpy()
        exp = oracle.dijkstra(n, g.src, g.dst, w, rows)
        if fp:
            got = got.astype(np.float64)
            np.testing.assert_array_equal(np.isinf(got), np.isinf(exp))
            f = np.isfinite(exp)
            assert (np.abs(got[f] - exp[f]) <= REL_TOL * exp[f]).all()
        else:
            np.testing.assert_array_equal(got.astype(np.int64), exp)


def test_gmm16k_int32_and_auto_whole_matrix(H):
    """gmm16k (n = 16384, 8 components): the int32 solve and the automatic-precision solve (bound, packed 16-bit
    rounds) equal the oracle's Dijkstra from every source, element by element."""
    g = gen.workload("gmm16k")
    W = dev(gen.dense_matrix(g.n, g.src, g.dst, g.w, dtype=np.int32))
    D = H.solve_t("int32", W)
    assert H.last_status() == 0
    A = H.solve_t("auto", W)
    assert H.last_status() == 0
    assert torch.equal(A, D)
    del A
    _whole_matrix_check(D, g)


def test_gmm16k_fp32_whole_matrix(H):
    """gmm16k with raw Euclidean fp32 weights: every row within 1e-4 relative of the float64 Dijkstra distances,
    the +inf set (pairs in different components) identical."""
    g = gen.workload("gmm16k_f32")
    W = dev(gen.dense_matrix(g.n, g.src, g.dst, g.w.astype(np.float32), dtype=np.float32))
    D = H.solve_t("fp32", W)
    assert H.last_status() == 0
    _whole_matrix_check(D, g, fp=True)


def test_fp32_negative_zero_weights_are_canonical(H):
    """A -0.0 weight is a zero-weight edge: stored as +0.0 by the input pass (the Phase-3 reduction compares fp32
    bit patterns as int32), so the result equals the same graph with +0.0 weights, in place and copied."""
    n = 300
    s, d, w = er_edges(n, seed=7, deg=4.0, wmax=30)
    wf = w.astype(np.float32)
    wf[::5] = 0.0
    Wp = gen.dense_matrix(n, s, d, wf, dtype=np.float32)
    Wn = Wp.copy()
    Wn[Wn == 0.0] = -0.0
    assert (np.signbit(Wn) & (Wn == 0)).sum() > n  # diagonal and the zero-weight edges are -0.0
    ref = H.solve_t("fp32", dev(Wp)).cpu().numpy()
    got = H.solve_t("fp32", dev(Wn)).cpu().numpy()
    assert H.last_status() == 0
    np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))
    Wi = dev(Wn)
    H.solve_t("fp32", Wi, Wi)  # in place
    np.testing.assert_array_equal(Wi.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    E = oracle.fw(Wp.astype(np.float64))
    np.testing.assert_array_equal(ref.astype(np.float64), E)  # integer-valued weights: exact


# ------------------------------------------------------------------ every round shape
@pytest.mark.parametrize("block_k", [32, 64, 128])
@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dt", ["int32", "u16", "fp32"])
def test_every_round_shape_matches_oracle(lib, block_k, variant, dt):
    n = 777
    s, d, w = er_edges(n, seed=block_k + 10 * variant, deg=3.0, wmax=40)
    E = expect_fw(gen.dense_matrix(n, s, d, w, dtype=np.int32))
    with lib.Handle(device=0, block_k=block_k, phase3_variant=variant) as h:
        if dt == "int32":
            D = h.solve_t(dt, dev(gen.dense_matrix(n, s, d, w, dtype=np.int32))).cpu().numpy().astype(np.int64)
        elif dt == "u16":
            D16 = h.solve_t(dt, dev(gen.dense_matrix(n, s, d, w, dtype=np.int16, inf=0x7FFF))).cpu().numpy()
            D = oracle.unpack_u16(D16.view(np.uint16)).astype(np.int64)
        else:
            Df = h.solve_t(dt, dev(gen.dense_matrix(n, s, d, w, dtype=np.float32))).cpu().numpy()
            D = np.where(np.isinf(Df), INF, Df.astype(np.float64)).astype(np.int64)  # small integers: exact
        np.testing.assert_array_equal(D, E)


@pytest.mark.parametrize("block_k", [32, 64, 128])
@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dt", ["int32", "u16", "fp32"])
def test_directed_every_phase3_kernel(lib, block_k, variant, dt):
    """Directed input (general mode) through every Phase-3 kernel.  The int32
    warp-specialized kernel reduces into the panel rows while other CTAs read
    them as operands; the result must still be exact."""
    n = 700
    s, d, w = er_edges(n, seed=block_k + variant, deg=3.0, wmax=60, directed=True)
    E = expect_fw(dense_directed(n, s, d, w))
    with lib.Handle(device=0, block_k=block_k, phase3_variant=variant) as h:
        if dt == "int32":
            D = h.solve_t(dt, dev(dense_directed(n, s, d, w))).cpu().numpy().astype(np.int64)
        elif dt == "u16":
            D16 = h.solve_t(dt, dev(dense_directed(n, s, d, w, dtype=np.int16, inf=0x7FFF))).cpu().numpy()
            D = oracle.unpack_u16(D16.view(np.uint16)).astype(np.int64)
        else:
            Df = h.solve_t(dt, dev(dense_directed(n, s, d, w, dtype=np.float32, inf=np.inf))).cpu().numpy()
            D = np.where(np.isinf(Df), INF, Df.astype(np.float64)).astype(np.int64)
        np.testing.assert_array_equal(D, E)


# ------------------------------------------------------------------ every round in one launch
# The single launch runs round k+1's Phase 1 / Phase 2 tasks in its work stream
# a few tile waves after the tiles they depend on; below ~2000 vertices they
# all fall at the end of a block, so these sizes are needed to run them between
# tiles (general and symmetric, directed too).
@pytest.mark.parametrize("symmetric,directed", [(2, False), (0, False), (0, True)])
def test_lookahead_midstream_int32_full_matrix(lib, symmetric, directed):
    n = 4100
    s, d, w = er_edges(n, seed=41 + symmetric + directed, deg=4.0, wmax=200, directed=directed)
    W = dense_directed(n, s, d, w) if directed else gen.dense_matrix(n, s, d, w, dtype=np.int32)
    E = oracle.dijkstra(n, s, d, w, np.arange(n), directed=directed)
    with lib.Handle(device=0, symmetric=symmetric, phase3_variant=5) as h:
        D = h.solve_t("int32", dev(W)).cpu().numpy().astype(np.int64)
        assert h.last_status() == 0
    np.testing.assert_array_equal(D, E)


@pytest.mark.parametrize("dt", ["u16", "fp32"])
def test_single_launch_general_mode_16bit_fp32_full_matrix(lib, dt):
    """Directed input (general mode), every round in one launch with its tasks between the tiles: the 16-bit tiles
    merge a loaded C and store it back, so each waits for its own previous round; the fp32 tiles leave by the
    int32 min-reduction on their bit patterns and may overlap the next round's; the whole matrix must equal the
    oracle's (Dijkstra from every source)."""
    n = 4100
    s, d, w = er_edges(n, seed=4100 + len(dt), deg=4.0, wmax=60, directed=True)
    E = oracle.dijkstra(n, s, d, w, np.arange(n), directed=True)
    with lib.Handle(device=0, phase3_variant=5) as h:
        if dt == "u16":
            D16 = h.solve_t(dt, dev(dense_directed(n, s, d, w, dtype=np.int16, inf=0x7FFF))).cpu().numpy()
            D = oracle.unpack_u16(D16.view(np.uint16)).astype(np.int64)
        else:
            Df = h.solve_t(dt, dev(dense_directed(n, s, d, w, dtype=np.float32, inf=np.inf))).cpu().numpy()
            D = np.where(np.isinf(Df), INF, Df.astype(np.float64)).astype(np.int64)  # small integers: exact
        assert h.last_status() == 0
    np.testing.assert_array_equal(D, E)


def test_lookahead_midstream_u16_sampled_rows(lib):
    n = 8200
    s, d, w = er_edges(n, seed=82, deg=4.0, wmax=60)
    W = gen.dense_matrix(n, s, d, w, dtype=np.int16, inf=0x7FFF)
    rows = np.sort(np.random.default_rng(8200).choice(n, size=512, replace=False))
    E = oracle.dijkstra(n, s, d, w, rows)
    with lib.Handle(device=0) as h:
        D = h.solve_t("u16", dev(W))
        assert h.last_status() == 0
        got = D[torch.from_numpy(rows).cuda().long()].cpu().numpy()
    np.testing.assert_array_equal(oracle.unpack_u16(got.view(np.uint16)).astype(np.int64), E)


def dense_on_device(n, s, d, w, dtype, inf, directed=False):
    """The dense matrix built on the device (no n x n host array at the largest sizes)."""
    tdt = {np.int32: torch.int32, np.int16: torch.int16}[dtype]
    W = torch.full((n, n), inf, dtype=tdt, device="cuda")
    src = np.asarray(s) if directed else np.concatenate([s, d])
    dst = np.asarray(d) if directed else np.concatenate([d, s])
    ww = np.asarray(w) if directed else np.concatenate([w, w])
    idx = torch.from_numpy(src.astype(np.int64) * n + dst.astype(np.int64)).cuda()
    W.view(-1).scatter_reduce_(0, idx, torch.from_numpy(ww).to(device="cuda", dtype=tdt), reduce="amin")
    W.fill_diagonal_(0)
    return W


@pytest.mark.parametrize("dt,n,directed", [("int32", 24000, False), ("int32", 24000, True), ("u16", 49000, False)])
def test_single_launch_top_of_default_range_sampled_rows(lib, dt, n, directed):
    """The largest sizes that take every round in one launch by default (int32 below 24576, packed 16-bit
    below 49152), ragged against the 128-row tiles: 128 seeded rows equal the oracle's Dijkstra rows, and the
    diagonal is zero."""
    s, d, w = er_edges(n, seed=n + directed, deg=4.0, wmax=60, directed=directed)
    inf = INF if dt == "int32" else 0x7FFF
    W = dense_on_device(n, s, d, w, np.int32 if dt == "int32" else np.int16, inf, directed)
    rows = np.sort(np.random.default_rng(n).choice(n, size=128, replace=False))
    with lib.Handle(device=0) as h:
        assert h.tuned_config(dt, n)[1] == 4  # every round in one launch
        h.solve_t(dt, W, W)  # in place
        assert h.last_status() == 0
    got = W[torch.from_numpy(rows).cuda().long()].cpu().numpy()
    assert bool((torch.diagonal(W) == 0).all())
    del W
    torch.cuda.empty_cache()
    if dt == "u16":
        got = oracle.unpack_u16(got.view(np.uint16))
    np.testing.assert_array_equal(got.astype(np.int64), oracle.dijkstra(n, s, d, w, rows, directed=directed))


# ------------------------------------------------------------------ symmetric mode
@pytest.mark.parametrize("symmetric", [0, 1, 2])
@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dt", ["int32", "u16", "fp32"])
@pytest.mark.parametrize("n", [65, 300, 1000])
def test_symmetric_mode_matches_oracle(lib, symmetric, variant, dt, n):
    """Undirected inputs: the symmetric mode (upper-triangle tiles + mirror),
    auto-detected (0), forced (1) or off (2), gives the oracle's matrix."""
    s, d, w = er_edges(n, seed=n + variant, deg=3.0, wmax=40)
    E = expect_fw(gen.dense_matrix(n, s, d, w, dtype=np.int32))
    with lib.Handle(device=0, phase3_variant=variant, symmetric=symmetric) as h:
        if dt == "int32":
            D = h.solve_t(dt, dev(gen.dense_matrix(n, s, d, w, dtype=np.int32))).cpu().numpy().astype(np.int64)
        elif dt == "u16":
            D16 = h.solve_t(dt, dev(gen.dense_matrix(n, s, d, w, dtype=np.int16, inf=0x7FFF))).cpu().numpy()
            D = oracle.unpack_u16(D16.view(np.uint16)).astype(np.int64)
        else:
            Df = h.solve_t(dt, dev(gen.dense_matrix(n, s, d, w, dtype=np.float32))).cpu().numpy()
            D = np.where(np.isinf(Df), INF, Df.astype(np.float64)).astype(np.int64)
        np.testing.assert_array_equal(D, E)


@pytest.mark.parametrize("block_k", [32, 64, 128])
def test_symmetric_mode_block_k_and_ld(lib, block_k):
    n, ld = 333, 340
    s, d, w = er_edges(n, seed=block_k, deg=3.0, wmax=500)
    W = gen.dense_matrix(n, s, d, w, dtype=np.int32, ld=ld)
    with lib.Handle(device=0, block_k=block_k, symmetric=1) as h:
        D = h.solve_t("int32", dev(W)).cpu().numpy()[:, :n]
    np.testing.assert_array_equal(D.astype(np.int64), expect_fw(W))


def test_auto_symmetric_detection_keeps_directed_exact(lib):
    n = 500
    s, d, w = er_edges(n, seed=99, deg=4.0, directed=True)
    W = dense_directed(n, s, d, w)
    with lib.Handle(device=0, symmetric=0) as h:
        D = h.solve_t("int32", dev(W)).cpu().numpy()
    np.testing.assert_array_equal(D.astype(np.int64), expect_fw(W))


# ------------------------------------------------------------------ degenerate graphs
def _solve_any(H, dt, n, s, d, w):
    if dt == "int32":
        return H.solve_t(dt, dev(gen.dense_matrix(n, s, d, w, dtype=np.int32))).cpu().numpy().astype(np.int64)
    if dt == "u16":
        D16 = H.solve_t(dt, dev(gen.dense_matrix(n, s, d, w, dtype=np.int16, inf=0x7FFF))).cpu().numpy()
        return oracle.unpack_u16(D16.view(np.uint16)).astype(np.int64)
    Df = H.solve_t(dt, dev(gen.dense_matrix(n, s, d, w, dtype=np.float32))).cpu().numpy()
    return np.where(np.isinf(Df), INF, Df.astype(np.float64)).astype(np.int64)


@pytest.mark.parametrize("dt", ["int32", "u16", "fp32"])
def test_zero_weight_edges(H, dt):
    n = 300
    s, d, w = er_edges(n, seed=21, deg=3.0, wmax=5)
    w = np.where(np.arange(w.shape[0]) % 3 == 0, 0, w)  # a third of the edges weigh 0
    E = expect_fw(gen.dense_matrix(n, s, d, w, dtype=np.int32))
    np.testing.assert_array_equal(_solve_any(H, dt, n, s, d, w), E)


@pytest.mark.parametrize("dt", ["int32", "u16", "fp32"])
def test_complete_graph_and_edgeless_graph(H, dt):
    n = 260
    iu, ju = np.triu_indices(n, 1)
    rng = np.random.default_rng(4)
    w = rng.integers(1, 50, size=iu.shape[0])
    E = expect_fw(gen.dense_matrix(n, iu, ju, w, dtype=np.int32))
    np.testing.assert_array_equal(_solve_any(H, dt, n, iu, ju, w), E)
    z = np.zeros(0, dtype=np.int64)
    E0 = np.full((n, n), INF, dtype=np.int64)
    np.fill_diagonal(E0, 0)
    np.testing.assert_array_equal(_solve_any(H, dt, n, z, z, z), E0)


@pytest.mark.parametrize("dt", ["int32", "u16", "fp32", "auto"])
def test_single_vertex(H, dt):
    np_dt = {"int32": np.int32, "auto": np.int32, "u16": np.int16, "fp32": np.float32}[dt]
    D = H.solve_t(dt, dev(np.zeros((1, 1), dtype=np_dt))).cpu().numpy()
    assert D.shape == (1, 1) and D[0, 0] == 0


# ------------------------------------------------------------------ pack / unpack through the C ABI
@pytest.mark.parametrize("n,lds,ldd", [(1, 1, 1), (5, 7, 8), (300, 301, 304), (1000, 1000, 1003)])
def test_pack_unpack_abi_match_oracle(lib, n, lds, ldd):
    """apsp_pack_u16 / apsp_unpack_u16 against oracle.pack_u16 / unpack_u16 with separate leading dimensions and
    the edge values 0, 1, 32766 (the largest finite 16-bit distance) and INF; padding columns stay untouched."""
    import ctypes
    rng = np.random.default_rng(n + lds + ldd)
    D32 = rng.integers(0, 32767, size=(n, n)).astype(np.int64)
    D32[rng.random((n, n)) < 0.2] = INF
    edge = np.array([0, 1, 32766, INF], dtype=np.int64)
    D32.reshape(-1)[: min(4, n * n)] = edge[: min(4, n * n)]
    src = np.full((n, lds), -5, dtype=np.int32)
    src[:, :n] = D32
    s_dev = dev(src)
    d_dev = torch.full((n, ldd), -3, dtype=torch.int16, device="cuda")
    L = lib.get_lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.apsp_pack_u16(ctypes.c_void_p(s_dev.data_ptr()), lds, ctypes.c_void_p(d_dev.data_ptr()), ldd, n,
                           stream) == 0
    got16 = d_dev.cpu().numpy().view(np.uint16)
    np.testing.assert_array_equal(got16[:, :n], oracle.pack_u16(D32.astype(np.int32)))
    assert (d_dev[:, n:] == -3).all()
    back = torch.full((n, lds), -9, dtype=torch.int32, device="cuda")
    assert L.apsp_unpack_u16(ctypes.c_void_p(d_dev.data_ptr()), ldd, ctypes.c_void_p(back.data_ptr()), lds, n,
                             stream) == 0
    got32 = back.cpu().numpy()
    np.testing.assert_array_equal(got32[:, :n], oracle.unpack_u16(got16[:, :n]))
    np.testing.assert_array_equal(got32[:, :n], D32)
    assert (back[:, n:] == -9).all()


# ------------------------------------------------------------------ upper-triangular storage
def _tri_dense_input(n, dt, seed):
    s, d, w = er_edges(n, seed=seed, deg=4.0, wmax=40)
    if dt == "int32":
        return gen.dense_matrix(n, s, d, w, dtype=np.int32), s, d, w
    if dt == "u16":
        return gen.dense_matrix(n, s, d, w, dtype=np.int16, inf=0x7FFF), s, d, w
    return gen.dense_matrix(n, s, d, w, dtype=np.float32), s, d, w


def _as_oracle_units(D, dt):
    if dt == "u16":
        return oracle.unpack_u16(D.view(np.uint16)).astype(np.int64)
    if dt == "fp32":
        return np.where(np.isinf(D), INF, D.astype(np.float64)).astype(np.int64)  # small integers: exact
    return D.astype(np.int64)


@pytest.mark.parametrize("dt", ["int32", "u16", "fp32"])
@pytest.mark.parametrize("n", [1, 2, 65, 129, 255, 257, 300, 700, 1300])
def test_tri_storage_solve_matches_oracle(lib, dt, n):
    """apsp_tri_from_dense -> apsp_solve_tri -> apsp_tri_to_dense / apsp_tri_rows: the full matrix equals the
    oracle's (Floyd-Warshall on the dense input), for sizes around the 128 / 256-element super-tiles."""
    W, *_ = _tri_dense_input(n, dt, seed=n + 17)
    E = expect_fw(_as_oracle_units(W, dt))
    with lib.Handle(device=0) as h:
        T = h.tri_from_dense(dt, dev(W))
        rows, ld, nbytes = lib.tri_layout(dt, n)
        assert tuple(T.shape) == (rows, ld) and T.numel() * T.element_size() == nbytes
        h.solve_tri(dt, T, n)
        assert h.last_status() == 0
        D = lib.tri_to_dense(dt, T, n).cpu().numpy()
        np.testing.assert_array_equal(_as_oracle_units(D, dt), E)
        pick = torch.tensor(sorted({0, n // 3, n // 2, n - 1}), dtype=torch.int64, device="cuda")
        R = lib.tri_rows(dt, T, n, pick).cpu().numpy()
        np.testing.assert_array_equal(_as_oracle_units(R, dt), E[pick.cpu().numpy()])


def test_tri_storage_from_edges_equals_dense_solve(lib):
    """The same graph from its edge list into upper-triangular storage and into a dense matrix: identical results
    (int32 and packed 16-bit), at a size with many super-tile rows in both halves of the folded rectangle."""
    n = 3000
    s, d, w = gen.er_graph(n, 77, avg_degree=8.0, wmax=200)
    with lib.Handle(device=0) as h:
        for dt, wdt in (("int32", np.int32), ("u16", np.int16)):
            src = torch.from_numpy(s.astype(np.int32)).cuda()
            dst = torch.from_numpy(d.astype(np.int32)).cuda()
            ww = torch.from_numpy(w.astype(wdt)).cuda()
            Dd = h.solve_edges(dt, src, dst, ww, n)
            T = h.tri_from_edges(dt, src, dst, ww, n)
            h.solve_tri(dt, T, n)
            assert h.last_status() == 0
            assert torch.equal(lib.tri_to_dense(dt, T, n), Dd)


def test_tri_storage_refuses_asymmetric_input(lib):
    n = 200
    s, d, w = er_edges(n, seed=5, deg=4.0, wmax=40, directed=True)
    W = dense_directed(n, s, d, w)
    with lib.Handle(device=0) as h:
        h.tri_from_dense("int32", dev(W))
        assert h.last_status() == lib.APSP_I32 + 1  # APSP_E_INVALID


def test_tri_storage_round_width_32_profiled_and_real_fp32(lib):
    """Upper-triangular storage with round width 32 and per-phase profiling on (int32, exact), and with real-valued
    fp32 weights (within the tolerance, +inf set identical)."""
    n = 700
    s, d, w = er_edges(n, seed=70, deg=4.0, wmax=90)
    with lib.Handle(device=0, block_k=32) as h:
        h.profile(True)
        T = h.tri_from_dense("int32", dev(gen.dense_matrix(n, s, d, w, dtype=np.int32)))
        h.solve_tri("int32", T, n)
        prof = h.profile_read()
        h.profile(False)
        assert h.last_status() == 0
        assert prof[3][0] == (n + 31) // 32 and prof[3][2] > 0  # one Phase-3 launch per round
        np.testing.assert_array_equal(lib.tri_to_dense("int32", T, n).cpu().numpy().astype(np.int64),
                                      expect_fw(gen.dense_matrix(n, s, d, w, dtype=np.int32)))
    rng = np.random.default_rng(71)
    wf = (rng.random(s.shape[0]) * 10 + 0.01).astype(np.float32)
    Wf = gen.dense_matrix(n, s, d, wf, dtype=np.float32)
    E = oracle.fw(Wf.astype(np.float64))
    with lib.Handle(device=0) as h:
        T = h.tri_from_dense("fp32", dev(Wf))
        h.solve_tri("fp32", T, n)
        assert h.last_status() == 0
        got = lib.tri_to_dense("fp32", T, n).cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(np.isinf(got), np.isinf(E))
    f = np.isfinite(E) & (E > 0)
    assert (np.abs(got[f] - E[f]) <= REL_TOL * E[f]).all()


def test_tri_storage_from_edges_duplicates_self_loops_and_bad_ids(lib):
    """The edge scatter into upper-triangular storage keeps the smaller weight of a duplicated edge (either
    orientation), ignores self loops, and reports a bad vertex id as APSP_E_INVALID."""
    n = 300
    s, d, w = er_edges(n, seed=72, deg=4.0, wmax=50)
    s2 = np.concatenate([s, d[:50], np.arange(20)])          # the reversed duplicates and 20 self loops
    d2 = np.concatenate([d, s[:50], np.arange(20)])
    w2 = np.concatenate([w, np.maximum(1, w[:50] - 3), np.full(20, 7)])
    E = expect_fw(gen.dense_matrix(n, s2, d2, w2, dtype=np.int32))
    with lib.Handle(device=0) as h:
        args = [torch.from_numpy(a.astype(np.int32)).cuda() for a in (s2, d2, w2)]
        T = h.tri_from_edges("int32", *args, n)
        h.solve_tri("int32", T, n)
        assert h.last_status() == 0
        np.testing.assert_array_equal(lib.tri_to_dense("int32", T, n).cpu().numpy().astype(np.int64), E)
        bad = [torch.tensor([0, 5], dtype=torch.int32, device="cuda"), torch.tensor([1, n + 3], dtype=torch.int32,
                                                                                    device="cuda"),
               torch.tensor([4, 4], dtype=torch.int32, device="cuda")]
        h.tri_from_edges("int32", *bad, n)
        assert h.last_status() == 1  # APSP_E_INVALID


# ------------------------------------------------------------------ round width 128
def _as_i64(dt, D):
    if dt == "u16":
        return oracle.unpack_u16(D.view(np.uint16)).astype(np.int64)
    if dt == "fp32":
        return np.where(np.isinf(D), INF, D.astype(np.float64)).astype(np.int64)  # small integers: exact
    return D.astype(np.int64)


def _dense_as(dt, n, s, d, w, directed):
    npdt, inf = {"int32": (np.int32, INF), "u16": (np.int16, 0x7FFF), "fp32": (np.float32, np.inf)}[dt]
    return gen.dense_matrix(n, s, d, w, dtype=npdt, inf=inf, directed=directed)


@pytest.mark.parametrize("dt", ["int32", "u16", "fp32"])
@pytest.mark.parametrize("variant", [1, 4])  # the per-tile kernel; the warp-specialized one (two stages per tile)
def test_round_width_128_ragged_sizes_both_modes(lib, dt, variant):
    """Round width 128: sizes whose last round ends inside the first or the second 64-step stage of a tile (or
    fills it), undirected (symmetric mode) and directed (general mode) inputs, against the oracle."""
    with lib.Handle(device=0, block_k=128, phase3_variant=variant) as h:
        assert h.tuned_config(dt, 300)[0] == 128
        for n in (1, 2, 63, 64, 65, 127, 128, 129, 191, 192, 193, 256, 300, 555):
            for directed in (False, True):
                s, d, w = er_edges(n, seed=n + 7 + directed, deg=3.0, wmax=50, directed=directed)
                W = _dense_as(dt, n, s, d, w, directed)
                E = expect_fw(_dense_as("int32", n, s, d, w, directed))
                got = _as_i64(dt, h.solve_t(dt, dev(W)).cpu().numpy())
                np.testing.assert_array_equal(got, E, err_msg=f"n={n} directed={directed}")


@pytest.mark.parametrize("dt", ["int32", "u16", "fp32"])
def test_round_width_128_upper_triangular_storage(lib, dt):
    """Upper-triangular storage solved with round width 128, unpacked and compared with the oracle, for sizes
    around the super-tile and round boundaries."""
    with lib.Handle(device=0, block_k=128) as h:
        for n in (1, 65, 129, 255, 257, 300, 700):
            s, d, w = er_edges(n, seed=3 * n + 1, deg=3.0, wmax=60)
            T = h.tri_from_dense(dt, dev(_dense_as(dt, n, s, d, w, False)))
            h.solve_tri(dt, T, n)
            assert h.last_status() == 0
            got = _as_i64(dt, lib.tri_to_dense(dt, T, n).cpu().numpy())
            np.testing.assert_array_equal(got, expect_fw(_dense_as("int32", n, s, d, w, False)), err_msg=f"n={n}")
