"""apsp_solve_i32_noalloc: the solve for callers that cannot allocate memory.

Some callers must not allocate device memory where they solve (they run
inside another framework's memory pool, or cannot afford the synchronization
an allocation can cause).  This entry point uses a fixed scratch array inside
the library instead of a handle's workspace.  The test calls it through the
C ABI twice in a row (on different sizes, so the second call runs on the
first call's leftover scratch contents) and compares each result with
apsp_solve_t, the existing entry point, exactly (integer distances).  The file
name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dense(n, seed):
    s, d, w = gen.er_graph(n, seed, avg_degree=6.0, wmax=1000)
    return torch.from_numpy(gen.dense_matrix(n, s, d, w, dtype=np.int32)).cuda()


def test_noalloc_solve_matches_solve_t_on_two_calls_in_a_row():
    import paper_1902_04446_gb300 as apsp
    L = apsp.get_lib()
    stream = torch.cuda.current_stream().cuda_stream
    Ws = [_dense(3001, 1), _dense(1000, 2)]  # larger first: the second call reuses a dirtier scratch
    outs = [torch.full_like(W, -1) for W in Ws]
    for W, D in zip(Ws, outs):
        n = W.shape[0]
        assert L.apsp_solve_i32_noalloc(ctypes.c_void_p(W.data_ptr()), n, n, ctypes.c_void_p(D.data_ptr()),
                                        ctypes.c_void_p(stream)) == 0
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
