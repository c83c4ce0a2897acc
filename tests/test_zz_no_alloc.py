"""apsp_solve_i32_noalloc: the solve for callers that cannot allocate memory.

Some callers must not allocate device memory where they solve (they run
inside another framework's memory pool, or cannot afford the synchronization
an allocation can cause).  This entry point uses a fixed scratch array inside
the library instead of a handle's workspace.  The tests call it through the
C ABI -- twice in a row on different sizes, so the second call runs on the
first call's leftover scratch contents; at the largest size it accepts, where
the panel fills the array exactly; with a padded leading dimension -- and
compare each result with apsp_solve_t, the existing entry point, exactly
(integer distances).  They also check that a warm call leaves the device's
free memory unchanged and that apsp_noalloc_status reports no timeout.  The
file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dense(n, seed, ld=None):
    s, d, w = gen.er_graph(n, seed, avg_degree=6.0, wmax=1000)
    return torch.from_numpy(gen.dense_matrix(n, s, d, w, dtype=np.int32, ld=ld)).cuda()


def _dense_on_device(n, seed):
    """A large ER adjacency matrix scattered on the device (no n x n host array)."""
    s, d, w = gen.er_graph(n, seed, avg_degree=8.0, wmax=1000)
    W = torch.full((n, n), 1073741823, dtype=torch.int32, device="cuda")
    src = torch.from_numpy(np.concatenate([s, d]).astype(np.int64)).cuda()
    dst = torch.from_numpy(np.concatenate([d, s]).astype(np.int64)).cuda()
    ww = torch.from_numpy(np.concatenate([w, w]).astype(np.int32)).cuda()
    W.view(-1).scatter_reduce_(0, src * n + dst, ww, reduce="amin")
    W.fill_diagonal_(0)
    return W


def _noalloc(L, W, D, stream):
    n, ld = W.shape[0], W.stride(0)
    return L.apsp_solve_i32_noalloc(ctypes.c_void_p(W.data_ptr()), n, ld, ctypes.c_void_p(D.data_ptr()),
                                    ctypes.c_void_p(stream))


def test_noalloc_solve_matches_solve_t_on_two_calls_in_a_row():
    import paper_1902_04446_gb300 as apsp
    L = apsp.get_lib()
    stream = torch.cuda.current_stream().cuda_stream
    Ws = [_dense(3001, 1), _dense(1000, 2)]  # larger first: the second call reuses a dirtier scratch
    outs = [torch.full_like(W, -1) for W in Ws]
    for W, D in zip(Ws, outs):
        assert _noalloc(L, W, D, stream) == 0
        assert L.apsp_noalloc_status(ctypes.c_void_p(stream)) == 0
    torch.cuda.synchronize()
    with apsp.Handle(device=0) as h:
        for W, D in zip(Ws, outs):
            ref = h.solve_t("int32", W)
            torch.cuda.synchronize()
            assert torch.equal(D, ref)


def test_noalloc_in_place_and_size_limit():
    import paper_1902_04446_gb300 as apsp
    L = apsp.get_lib()
    W = _dense(513, 3)
    with apsp.Handle(device=0) as h:
        ref = h.solve_t("int32", W)
    n = W.shape[0]
    assert L.apsp_solve_i32_noalloc(ctypes.c_void_p(W.data_ptr()), n, n, ctypes.c_void_p(W.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert torch.equal(W, ref)
    big = apsp.lib.apsp_solve_i32_noalloc
    # beyond the static scratch: refused before anything is touched
    assert big(ctypes.c_void_p(W.data_ptr()), 16385, 16385, ctypes.c_void_p(W.data_ptr()), None) == 4
    assert big(None, 10, 10, None, None) == 1


def test_noalloc_padded_leading_dimension():
    import paper_1902_04446_gb300 as apsp
    L = apsp.get_lib()
    n = 1300
    W = _dense(n, 4, ld=n + 4)[:, :n]  # rows of n + 4 elements, the first n used
    assert W.stride(0) == n + 4
    Dfull = torch.full((n, n + 4), -7, dtype=torch.int32, device="cuda")
    D = Dfull[:, :n]
    stream = torch.cuda.current_stream().cuda_stream
    assert _noalloc(L, W, D, stream) == 0
    assert L.apsp_noalloc_status(ctypes.c_void_p(stream)) == 0
    with apsp.Handle(device=0) as h:
        ref = h.solve_t("int32", W, torch.empty((n, n + 4), dtype=torch.int32, device="cuda")[:, :n])
    torch.cuda.synchronize()
    assert torch.equal(D, ref)
    assert bool((Dfull[:, n:] == -7).all())  # the padding columns are never written


def test_noalloc_at_the_size_limit_and_no_device_memory_taken():
    """n = APSP_NOALLOC_MAX_N with ld = n: the round panel fills the scratch array exactly.  A warm call (same size,
    so no code is loaded for it) must leave the device's free memory exactly as it was."""
    import paper_1902_04446_gb300 as apsp
    L = apsp.get_lib()
    n = 16384
    W = _dense_on_device(n, 5)
    D = torch.empty_like(W)
    stream = torch.cuda.current_stream().cuda_stream
    assert _noalloc(L, W, D, stream) == 0  # first call at this size: may load code
    assert L.apsp_noalloc_status(ctypes.c_void_p(stream)) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _noalloc(L, W, D, stream) == 0
    assert L.apsp_noalloc_status(ctypes.c_void_p(stream)) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    with apsp.Handle(device=0) as h:
        ref = h.solve_t("int32", W)
    torch.cuda.synchronize()
    assert torch.equal(D, ref)
