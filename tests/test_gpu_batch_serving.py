"""Batched persistent solves and the request loop, against the oracle (GPU).

Bit-exact for every graph, alone and in a mix; admission against a memory
budget; queue limits; cancellation; bounded device waits that report a
timeout status instead of hanging.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
INF = oracle.INF32


@pytest.fixture(scope="module")
def H(lib):
    h = lib.Handle(device=0)
    yield h
    h.close()


def er_dense(n, seed, deg=6.0, wmax=1000):
    s, d, w = gen.er_graph(n, seed, avg_degree=deg, wmax=wmax) if n > 1 else (np.zeros(0, np.int64),) * 3
    return gen.dense_matrix(n, s, d, w, dtype=np.int32)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SIZES = [1, 2, 64, 65, 100, 257, 513, 700, 1000]


def test_solve_batch_mixed_sizes_bit_exact(H):
    Ws = [er_dense(n, 100 + n) for n in SIZES]
    Ds = H.solve_batch([dev(W) for W in Ws])
    assert H.last_status() == 0
    for W, D in zip(Ws, Ds):
        np.testing.assert_array_equal(D.cpu().numpy().astype(np.int64), oracle.fw(W.astype(np.int64)))


def test_solve_batch_equals_alone_and_handles_in_place_and_empty(H):
    Ws = [er_dense(n, 7 * n) for n in (300, 129, 640)]
    alone = [H.solve_t("int32", dev(W)).cpu() for W in Ws]
    ins = [dev(W) for W in Ws]
    H.solve_batch(ins, ins)  # in place
    for a, b in zip(alone, ins):
        assert torch.equal(a, b.cpu())
    assert H.solve_batch([]) == []
    z = torch.zeros((0, 0), dtype=torch.int32, device="cuda")
    H.solve_batch([z, dev(Ws[1])])


def test_bounded_wait_reports_timeout_and_context_survives(H):
    """The batched kernel and the all-rounds persistent launch each wait on a flag that nothing sets, give up
    after the spin limit and report APSP_E_TIMEOUT; afterwards both kernels solve exactly on the same context."""
    import time
    t0 = time.perf_counter()
    assert H.check_bounded_wait(1 << 10) == 7  # APSP_E_TIMEOUT
    assert time.perf_counter() - t0 < 30.0  # the CTAs stop together, not one full wait limit after another
    W = er_dense(200, 3)
    D = H.solve_t("int32", dev(W))
    np.testing.assert_array_equal(D.cpu().numpy().astype(np.int64), oracle.fw(W.astype(np.int64)))
    n = 6200  # every round in one launch by default from n = 6144
    s, d, w = gen.er_graph(n, 31, avg_degree=6.0)
    D = H.solve_t("int32", dev(gen.dense_matrix(n, s, d, w, dtype=np.int32))).cpu().numpy()
    rows = np.array([0, 1, 1550, 3099])
    np.testing.assert_array_equal(D[rows].astype(np.int64), oracle.dijkstra(n, s, d, w, rows))


def test_serving_mixed_equals_alone_and_oracle(H):
    reqs = [gen.serving_request(1000 + i, n_lo=64, n_hi=900) for i in range(24)]
    Ws = [gen.dense_matrix(r.n, r.src, r.dst, r.w, dtype=np.int32) for r in reqs]
    # half device, half host (pinned and pageable) inputs
    ins = [dev(W) if i % 2 == 0 else (torch.from_numpy(W).pin_memory() if i % 4 == 1 else torch.from_numpy(W))
           for i, W in enumerate(Ws)]
    tickets = [H.submit(x) for x in ins]
    outs = []
    for t, W in zip(tickets, Ws):
        assert H.wait(t, 60000) == 0
        st, ptr, rc = H.poll(t)
        assert st == 3 and rc == 0 and ptr
        out = torch.empty((W.shape[0], W.shape[0]), dtype=torch.int32, device="cuda")
        H.fetch(t, out)
        torch.cuda.synchronize()
        outs.append(out.cpu())
        assert H.release(t) == 0
    for W, o in zip(Ws, outs):
        alone = H.solve_t("int32", dev(W)).cpu()
        assert torch.equal(o, alone)
        np.testing.assert_array_equal(o.numpy().astype(np.int64), oracle.fw(W.astype(np.int64)))


def test_serving_large_requests_on_round_kernels(H):
    """Requests with n >= 1536 take their own group on the per-round kernels, an undirected one in
    symmetric mode and a directed one on the general path; mixed with small batched requests, each result equals
    the same matrix solved alone and the oracle's (Dijkstra from every source)."""
    rng = np.random.default_rng(1536)
    cases = []
    for n, directed in ((1600, False), (1700, True), (300, False), (2100, False), (500, True)):
        m = int(4 * n)
        s = rng.integers(0, n, m); d = rng.integers(0, n, m); keep = s != d
        s, d = s[keep], d[keep]
        w = rng.integers(1, 500, s.shape[0])
        W = gen.dense_matrix(n, s, d, w, dtype=np.int32, directed=directed)
        cases.append((W, s, d, w, directed))
    tickets = [H.submit(dev(W)) for W, *_ in cases]
    for t, (W, s, d, w, directed) in zip(tickets, cases):
        n = W.shape[0]
        assert H.wait(t, 120000) == 0
        st, ptr, rc = H.poll(t)
        assert st == 3 and rc == 0 and ptr
        out = torch.empty((n, n), dtype=torch.int32, device="cuda")
        H.fetch(t, out)
        torch.cuda.synchronize()
        assert H.release(t) == 0
        alone = H.solve_t("int32", dev(W))
        assert torch.equal(out, alone)
        exp = oracle.dijkstra(n, s, d, w, np.arange(n), directed=directed)
        np.testing.assert_array_equal(out.cpu().numpy().astype(np.int64), exp)


def test_serving_budget_admission_busy_cancel(lib):
    big = er_dense(1000, 5)
    small = [er_dense(n, n) for n in (300, 320, 340)]  # each larger than the big one's panel buffer
    budget = 1000 * 1000 * 4 + 64 * 1024 * 4 + 256  # exactly the big request
    with lib.Handle(device=0, memory_budget=budget, queue_depth=2) as h:
        with pytest.raises(lib.ApspError) as ei:
            h.submit(dev(er_dense(1100, 1)))  # larger than the whole budget
        assert ei.value.name == "APSP_E_NOMEM"
        tb = h.submit(dev(big))
        assert h.wait(tb, 60000) == 0
        # the big matrix is held until released: the small ones stay queued
        t1 = h.submit(dev(small[0]))
        t2 = h.submit(dev(small[1]))
        with pytest.raises(lib.ApspError) as ei:
            h.submit(dev(small[2]))
        assert ei.value.name == "APSP_E_BUSY"
        import time
        time.sleep(0.05)
        assert h.poll(t1)[0] == 0 and h.poll(t2)[0] == 0  # QUEUED
        assert h.cancel(t2) == 0
        st, _, rc = h.poll(t2)
        assert st == 4 and rc == 8  # ERROR, APSP_E_CANCELLED
        assert h.release(tb) == 0  # memory returns: t1 is admitted and runs
        assert h.wait(t1, 60000) == 0
        out = torch.empty((300, 300), dtype=torch.int32, device="cuda")
        h.fetch(t1, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy().astype(np.int64), oracle.fw(small[0].astype(np.int64)))
        h.release(t1)
        h.release(t2)


def test_serving_reports_input_errors_per_request(H):
    good1, good2 = er_dense(120, 11), er_dense(90, 12)
    bad = er_dense(90, 2)
    bad[5, 7] = -1
    ts = [H.submit(dev(x)) for x in (good1, bad, good2)]  # usually admitted as one group
    assert [H.wait(t, 60000) for t in ts] == [0, 1, 0]  # only the bad one is APSP_E_INVALID
    st, _, rc = H.poll(ts[1])
    assert st == 4 and rc == 1
    for t, W in ((ts[0], good1), (ts[2], good2)):
        out = torch.empty(W.shape, dtype=torch.int32, device="cuda")
        H.fetch(t, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy().astype(np.int64), oracle.fw(W.astype(np.int64)))
    for t in ts:
        H.release(t)


@pytest.mark.parametrize("dtype,n,p3", [
    ("int32", 2048, 3), ("int32", 6143, 3), ("int32", 6144, 4), ("int32", 16384, 4), ("int32", 24575, 4),
    ("int32", 24576, 3), ("int32", 65536, 3), ("fp32", 5120, 3), ("fp32", 16384, 4), ("fp32", 32768, 3),
    ("u16", 6143, 3), ("u16", 6144, 4), ("u16", 32768, 4), ("u16", 49151, 4), ("u16", 49152, 3),
    ("u16", 262144, 3)])
def test_default_phase3_kernel_by_n_and_dtype(lib, dtype, n, p3):
    """Untuned, the handle takes every round in one launch (kernel 4) for mid-size n and one launch per round
    (kernel 3) below and above; packed 16-bit, with half the tiles per round, keeps the single launch longer.
    Large n in packed 16-bit and fp32 runs 128-wide rounds, everything else 64-wide."""
    bk = 128 if dtype != "int32" and p3 == 3 and n >= 6144 else 64
    with lib.Handle(device=0) as h:
        assert h.tuned_config(dtype, n) == (bk, p3)


def test_autotune_cache_and_bit_exact_with_every_shape(lib, tmp_path):
    cache = str(tmp_path / "tune.json")
    with lib.Handle(device=0) as h:
        table = h.autotune("int32", 512, cache)
        assert set(table) == {128, 256, 512}
        assert all(bk in (32, 64, 128) and p3 in (0, 1, 2, 3, 4) for bk, p3 in table.values())
        assert all(p3 in (0, 3) for bk, p3 in table.values() if bk == 128)
    import json
    entries = json.load(open(cache))["entries"]
    assert {e["n"] for e in entries} == {128, 256, 512} and all(e["ms"] > 0 for e in entries)
    with lib.Handle(device=0) as h2:
        assert h2.autotune("int32", 512, cache) == table  # loaded from the cache
    # every round shape gives the same exact answer
    W = er_dense(300, 77)
    E = oracle.fw(W.astype(np.int64))
    for bk in (32, 64, 128):
        with lib.Handle(device=0, block_k=bk) as hb:
            assert hb.tuned_config("int32", 300)[0] == bk
            for dt, Wx in (("int32", W), ("u16", None)):
                if dt == "u16":
                    Wx = np.where(W >= INF, 0x7FFF, W).astype(np.int16)
                    if E[E < INF].max() >= 0x7FFF:
                        continue
                D = hb.solve_t(dt, dev(Wx)).cpu().numpy()
                if dt == "u16":
                    D = oracle.unpack_u16(D.view(np.uint16))
                np.testing.assert_array_equal(D.astype(np.int64), E)


@pytest.mark.parametrize("n", [31, 100, 257, 1000])
def test_block_k_32_matches_oracle(lib, n):
    W = er_dense(n, 5 + n)
    with lib.Handle(device=0, block_k=32) as h:
        D = h.solve_t("int32", dev(W)).cpu().numpy()
        np.testing.assert_array_equal(D.astype(np.int64), oracle.fw(W.astype(np.int64)))
        Wf = np.where(W >= INF, np.inf, W).astype(np.float32)
        Df = h.solve_t("fp32", dev(Wf)).cpu().numpy()
        E = oracle.fw(W.astype(np.int64)).astype(np.float64)
        E[E >= INF] = np.inf
        np.testing.assert_array_equal(Df.astype(np.float64), E)  # small integers: exact in fp32


def test_serving_states_admitted_then_running(lib):
    """apsp_poll walks QUEUED -> ADMITTED (input copy in flight) -> RUNNING (W copied, rounds running) -> DONE, never
    backwards.  Large pinned host inputs make the copy long enough to be seen; the handle skips the symmetry check
    (symmetric = 2), which would otherwise wait for the copy inside admission."""
    seen_admitted = False
    with lib.Handle(device=0, symmetric=2) as h:
        for i in range(4):
            W = torch.from_numpy(er_dense(4000, 40 + i)).pin_memory()
            t = h.submit(W)
            states = []
            while True:
                st, _, rc = h.poll(t)
                assert rc == 0
                if not states or states[-1] != st:
                    states.append(st)
                if st == 3:
                    break
            assert states == sorted(states), states
            seen_admitted |= 1 in states
            assert 2 in states or states[-1] == 3
            out = torch.empty((4000, 4000), dtype=torch.int32, device="cuda")
            h.fetch(t, out)
            torch.cuda.synchronize()
            assert h.release(t) == 0
            assert torch.equal(out, h.solve_t("int32", W.cuda()))
    assert seen_admitted


def test_serving_auto_requests_equal_int32_and_oracle(H):
    """apsp_request.dtype = APSP_AUTO: a large request whose 16-bit bound holds runs its rounds in packed 16-bit,
    one whose bound fails (a long heavy path) and the small ones run in int32; every result is the int32 matrix,
    equal to the same graph solved alone and to the oracle."""
    cases = []
    for n, seed, wmax in ((2000, 71, 100), (400, 72, 1000), (1700, 73, 100)):
        s, d, w = gen.er_graph(n, seed, avg_degree=8.0, wmax=wmax)
        cases.append((gen.dense_matrix(n, s, d, w, dtype=np.int32), s, d, w))
    n = 1600  # path with weight 1000: distances up to 1.6e6, the 16-bit bound fails
    s = np.arange(n - 1)
    d = s + 1
    w = np.full(n - 1, 1000)
    cases.append((gen.dense_matrix(n, s, d, w, dtype=np.int32), s, d, w))
    W0 = dev(cases[0][0])
    b, ok = H.int16_bound(W0)
    assert ok, b  # the first large request does take the packed path
    tickets = [H.submit(dev(W), dtype="auto") for W, *_ in cases]
    for t, (W, s, d, w) in zip(tickets, cases):
        n = W.shape[0]
        assert H.wait(t, 120000) == 0
        out = torch.empty((n, n), dtype=torch.int32, device="cuda")
        H.fetch(t, out)
        torch.cuda.synchronize()
        assert H.release(t) == 0
        assert torch.equal(out, H.solve_t("int32", dev(W)))
        np.testing.assert_array_equal(out.cpu().numpy().astype(np.int64), oracle.dijkstra(n, s, d, w, np.arange(n)))
    with pytest.raises(Exception):
        H.submit(dev(cases[1][0]), dtype="fp32")


def test_serving_lone_requests_run_alone_and_exact(lib):
    """A request that finds the server idle runs alone on the per-round kernels (like a one-at-a-time solve): one
    request at a time, small and directed ones included, each equal to the oracle."""
    rng = np.random.default_rng(77)
    with lib.Handle(device=0) as h:
        for n, directed in ((90, False), (333, True), (700, False), (1100, True)):
            m = 4 * n
            s = rng.integers(0, n, m); d = rng.integers(0, n, m); keep = s != d
            s, d = s[keep], d[keep]
            w = rng.integers(1, 300, s.shape[0])
            W = gen.dense_matrix(n, s, d, w, dtype=np.int32, directed=directed)
            t = h.submit(dev(W) if n % 2 == 0 else torch.from_numpy(W))
            assert h.wait(t, 60000) == 0
            out = torch.empty((n, n), dtype=torch.int32, device="cuda")
            h.fetch(t, out)
            torch.cuda.synchronize()
            assert h.release(t) == 0
            np.testing.assert_array_equal(out.cpu().numpy().astype(np.int64),
                                          oracle.dijkstra(n, s, d, w, np.arange(n), directed=directed))
