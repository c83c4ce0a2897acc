"""Pins for the CPU oracle (no GPU needed).

The paper prints no distance values, so the oracle is tied to things other than
itself: brute-force path enumeration, closed forms, invariants that
characterise the shortest-path metric, the paper's own alternative routes
(Alg. 1 repeated squaring, Alg. 2 per-k rank-1 updates), and SciPy's csgraph
routines.  Every check below runs on the CPU in seconds.
"""
import numpy as np
import pytest

import gen
import oracle
from tests import pins

INF = oracle.INF32


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("directed", [False, True])
def test_fw_matches_brute_force_tiny(seed, directed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 9))
    p = [0.2, 0.4, 0.7, 1.0][seed % 4]
    edges = pins.random_graph(rng, n, p, wmax=20, directed=directed, zero_ok=(seed % 3 == 0))
    W = pins.dense(n, edges, directed)
    expect = pins.brute_force(n, edges, directed)
    np.testing.assert_array_equal(oracle.fw(W), expect)
    if edges:
        s = np.array([e[0] for e in edges]); d = np.array([e[1] for e in edges]); w = np.array([e[2] for e in edges])
    else:
        s = d = w = np.zeros(0, dtype=np.int64)
    np.testing.assert_array_equal(oracle.dijkstra(n, s, d, w, np.arange(n), directed=directed), expect)


# ---------------------------------------------------------------- closed forms
def _solve_both(n, s, d, w):
    W = gen.dense_matrix(n, s, d, w, dtype=np.int64)
    D = oracle.fw(W)
    R = oracle.dijkstra(n, s, d, w, np.arange(n))
    np.testing.assert_array_equal(D, R)
    return D


def test_path_graph():
    n, w = 37, 7
    s = np.arange(n - 1); d = s + 1
    D = _solve_both(n, s, d, np.full(n - 1, w))
    i, j = np.indices((n, n))
    np.testing.assert_array_equal(D, np.abs(i - j) * w)


def test_unit_grid_is_manhattan():
    r, c = 6, 9
    idx = np.arange(r * c).reshape(r, c)
    s = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    d = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    D = _solve_both(r * c, s, d, np.ones_like(s))
    rr, cc = np.divmod(np.arange(r * c), c)
    np.testing.assert_array_equal(D, np.abs(rr[:, None] - rr[None, :]) + np.abs(cc[:, None] - cc[None, :]))


def test_cycle():
    n, w = 25, 3
    s = np.arange(n); d = (s + 1) % n
    D = _solve_both(n, s, d, np.full(n, w))
    i, j = np.indices((n, n))
    k = np.abs(i - j)
    np.testing.assert_array_equal(D, w * np.minimum(k, n - k))


def test_complete_graph():
    n, w = 11, 5
    iu, ju = np.triu_indices(n, 1)
    D = _solve_both(n, iu, ju, np.full(iu.shape, w))
    np.testing.assert_array_equal(D, w * (1 - np.eye(n, dtype=np.int64)))


def test_star():
    n, w = 10, 4
    s = np.zeros(n - 1, dtype=np.int64); d = np.arange(1, n)
    D = _solve_both(n, s, d, np.full(n - 1, w))
    expect = np.full((n, n), 2 * w, dtype=np.int64)
    expect[0, :] = w; expect[:, 0] = w
    np.fill_diagonal(expect, 0)
    np.testing.assert_array_equal(D, expect)


def test_two_components_are_inf_across():
    a = 6
    s = np.concatenate([np.arange(a - 1), a + np.arange(a - 1)])
    d = s + 1
    D = _solve_both(2 * a, s, d, np.full(s.shape, 2))
    assert (D[:a, a:] == INF).all() and (D[a:, :a] == INF).all()
    i, j = np.indices((a, a))
    np.testing.assert_array_equal(D[:a, :a], 2 * np.abs(i - j))
    np.testing.assert_array_equal(D[a:, a:], 2 * np.abs(i - j))


def test_single_vertex_and_empty():
    np.testing.assert_array_equal(oracle.fw(np.zeros((1, 1), dtype=np.int64)), [[0]])
    assert oracle.fw(np.zeros((0, 0), dtype=np.int64)).shape == (0, 0)


def test_fp64_path_graph():
    n = 20
    s = np.arange(n - 1); d = s + 1; w = np.full(n - 1, 0.25)
    W = gen.dense_matrix(n, s, d, w, dtype=np.float64)
    D = oracle.fw(W)
    i, j = np.indices((n, n))
    np.testing.assert_allclose(D, 0.25 * np.abs(i - j), rtol=0, atol=1e-12)


# ---------------------------------------------------------------- invariants
def _check_metric_invariants(D, W, s, d, n):
    # symmetry and zero diagonal
    np.testing.assert_array_equal(D, D.T)
    assert (np.diag(D) == 0).all()
    # d(i,j) <= w(i,j)
    assert (D <= W).all()
    # INF exactly on different-component pairs
    lab = oracle.components(n, s, d)
    same = lab[:, None] == lab[None, :]
    assert ((D >= INF) == ~same).all()
    # triangle inequality d(i,j) <= d(i,k) + d(k,j) over every k
    Df = np.where(D >= INF, np.inf, D.astype(np.float64))
    for k in range(n):
        assert (Df <= Df[:, k][:, None] + Df[k, :][None, :]).all()
    # Bellman equations: every finite off-diagonal d(i,j) equals
    # min over neighbours m of i of w(i,m) + d(m,j); with positive weights this
    # fixed point is unique, so together with the above it pins the metric.
    Wf = np.where(W >= INF, np.inf, W.astype(np.float64))
    np.fill_diagonal(Wf, np.inf)
    bell = np.min(Wf[:, :, None] + Df[None, :, :], axis=1)
    off = ~np.eye(n, dtype=bool) & np.isfinite(Df)
    np.testing.assert_array_equal(Df[off], bell[off])


def test_invariants_on_swiss_roll_512():
    g = gen.workload("roll512")
    W = gen.dense_matrix(g.n, g.src, g.dst, g.w, dtype=np.int64)
    D = oracle.fw(W)
    _check_metric_invariants(D, W, g.src, g.dst, g.n)


def test_invariants_on_disconnected_er():
    rng = np.random.default_rng(7)
    n = 160
    edges = pins.random_graph(rng, n, 0.012, wmax=50)
    s = np.array([e[0] for e in edges]); d = np.array([e[1] for e in edges]); w = np.array([e[2] for e in edges])
    W = gen.dense_matrix(n, s, d, w, dtype=np.int64)
    D = oracle.fw(W)
    assert (D >= INF).any()  # the case of interest: several components
    _check_metric_invariants(D, W, s, d, n)


# ---------------------------------------------------------------- independent routes
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fw_equals_alg1_alg2_dijkstra(seed):
    rng = np.random.default_rng(100 + seed)
    n = [48, 97, 130][seed]
    edges = pins.random_graph(rng, n, 3.0 / n, wmax=100)
    W = pins.dense(n, edges)
    s = np.array([e[0] for e in edges]); d = np.array([e[1] for e in edges]); w = np.array([e[2] for e in edges])
    D = oracle.fw(W)
    np.testing.assert_array_equal(D, pins.repeated_squaring(W))
    np.testing.assert_array_equal(D, pins.rank1_fw(W))
    np.testing.assert_array_equal(D, oracle.dijkstra(n, s, d, w, np.arange(n)))


def test_matches_scipy_csgraph():
    sp = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sps
    g = gen.workload("roll512")
    A = sps.coo_matrix((g.w.astype(np.float64), (g.src, g.dst)), shape=(g.n, g.n)).tocsr()
    ref = sp.floyd_warshall(A, directed=False)
    W = gen.dense_matrix(g.n, g.src, g.dst, g.w, dtype=np.int64)
    D = oracle.fw(W)
    np.testing.assert_array_equal(np.where(np.isinf(ref), INF, ref).astype(np.int64), D)
    ref2 = sp.dijkstra(A, directed=False, indices=[0, 17, 511])
    np.testing.assert_array_equal(np.where(np.isinf(ref2), INF, ref2).astype(np.int64),
                                  oracle.dijkstra(g.n, g.src, g.dst, g.w, [0, 17, 511]))


def test_fp64_matches_scipy():
    sp = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sps
    rng = np.random.default_rng(3)
    pts = gen.gaussian_mixture(300, 5, dim=4, components=3)
    s, d, dist = gen.knn_edges(pts, 5)
    w = dist.astype(np.float32).astype(np.float64)
    A = sps.coo_matrix((w, (s, d)), shape=(300, 300)).tocsr()
    ref = sp.floyd_warshall(A, directed=False)
    W = gen.dense_matrix(300, s, d, w, dtype=np.float64)
    D = oracle.fw(W)
    np.testing.assert_allclose(D, ref, rtol=1e-12, atol=0)
    R = oracle.dijkstra(300, s, d, w, np.arange(300))
    np.testing.assert_allclose(R, ref, rtol=1e-12, atol=0)
    assert rng is not None


# ---------------------------------------------------------------- min-plus product
def test_minplus_against_broadcast_definition():
    rng = np.random.default_rng(11)
    m, kk, nn = 13, 7, 9
    A = rng.integers(0, 50, size=(m, kk)); B = rng.integers(0, 50, size=(kk, nn)); C = rng.integers(0, 120, size=(m, nn))
    A[rng.random(A.shape) < 0.3] = INF
    B[rng.random(B.shape) < 0.3] = INF
    got = oracle.minplus(A, B, C)
    # brute force over t, INF absorbing
    exp = C.copy()
    for i in range(m):
        for j in range(nn):
            for t in range(kk):
                if A[i, t] < INF and B[t, j] < INF:
                    exp[i, j] = min(exp[i, j], A[i, t] + B[t, j])
    np.testing.assert_array_equal(got, exp)
    # identity: the min-plus identity (0 diagonal, INF elsewhere) leaves B unchanged
    I0 = np.full((kk, kk), INF, dtype=np.int64); np.fill_diagonal(I0, 0)
    np.testing.assert_array_equal(oracle.minplus(I0, B, np.full((kk, nn), INF)), B)


def test_minplus_fp64_against_broadcast_definition():
    """The float product with +inf entries, against the definition written with numpy broadcasting."""
    rng = np.random.default_rng(12)
    m, kk, nn = 11, 6, 8
    A = rng.random((m, kk)) * 10; B = rng.random((kk, nn)) * 10; C = rng.random((m, nn)) * 25
    A[rng.random(A.shape) < 0.3] = np.inf
    B[rng.random(B.shape) < 0.3] = np.inf
    C[rng.random(C.shape) < 0.2] = np.inf
    exp = np.minimum(C, (A[:, :, None] + B[None, :, :]).min(axis=1))
    np.testing.assert_array_equal(oracle.minplus(A, B, C), exp)


def test_fw_k_slices_compose():
    """Running the outer loop in two slices equals one full run (used by the CPU baseline)."""
    g = gen.workload("roll512")
    W = gen.dense_matrix(g.n, g.src, g.dst, g.w, dtype=np.int64)
    a = oracle.fw(W, 0, 200)
    b = oracle.fw(a, 200, g.n)
    np.testing.assert_array_equal(b, oracle.fw(W))


# ---------------------------------------------------------------- int16 bound and packing
def test_int16_bound_closed_form_path():
    n, w = 40, 9
    s = np.arange(n - 1); d = s + 1
    bound, ok = oracle.int16_bound(n, s, d, np.full(n - 1, w))
    # root = vertex 0, ecc(0) = (n-1) w
    assert bound == 2 * (n - 1) * w and ok
    bound, ok = oracle.int16_bound(n, s, d, np.full(n - 1, 500))
    assert bound == 2 * 39 * 500 and not ok


def test_int16_bound_closed_form_two_components():
    """Two disjoint weighted paths: the bound is the larger of the two components' 2 ecc(root), each root the
    component's smallest vertex, and unreachable pairs do not enter it."""
    s = np.array([0, 1, 2, 3, 5, 6, 7]); d = s + 1
    w = np.array([3, 3, 3, 3, 7, 7, 7])
    bound, ok = oracle.int16_bound(9, s, d, w)  # vertex 4 ends path A; vertex 8 ends path B
    assert bound == max(2 * 4 * 3, 2 * 3 * 7) and ok


def test_int16_bound_is_sound_on_er():
    rng = np.random.default_rng(5)
    n = 120
    edges = pins.random_graph(rng, n, 0.02, wmax=300)
    s = np.array([e[0] for e in edges]); d = np.array([e[1] for e in edges]); w = np.array([e[2] for e in edges])
    bound, _ = oracle.int16_bound(n, s, d, w)
    D = oracle.fw(gen.dense_matrix(n, s, d, w, dtype=np.int64))
    fin = D[D < INF]
    assert fin.max() <= bound  # the bound really bounds every finite distance


def test_pack_roundtrip_and_inf_mapping():
    D = np.array([[0, 5, INF], [5, 0, 32766], [INF, 32766, 0]], dtype=np.int32)
    P = oracle.pack_u16(D)
    assert P.dtype == np.uint16 and P[0, 2] == 0x7FFF and P[1, 2] == 32766
    np.testing.assert_array_equal(oracle.unpack_u16(P), D)
    with pytest.raises(ValueError):
        oracle.pack_u16(np.array([[0, 32767]], dtype=np.int32))
