#!/usr/bin/env python
"""Benchmark of the blocked Floyd-Warshall APSP library on one GB300.

Metric: APSP relaxations per second, n^3 / t (the paper's "ops" of Sec. 5.4),
reported in GRelax/s, for int32 and for packed 16-bit distances.  The default
workload is roll64k: the n = 65536 Swiss-roll kNN graph (int32 weights
max(1, rint(4 d))), the size at which both element types are measured.  One
step = one apsp_solve of the whole workload matrix (ingest, symmetry check,
q rounds of Phase 1 / 2 / 3, mirror pass), inputs resident in HBM; the graph
is undirected, so the default path runs the symmetric mode (about half the
relaxations).  The matrix (17.2 GB) is larger than L2, so no flush is needed.

Printed JSON line (rank 0): the headline int32 number with the live Phase-3
roofline, the packed-16-bit number on the same graph and steps (automatic
precision selection: bound + pack + u16x2 rounds + unpack), the end-to-end
number through host buffers on the same graph and steps, clocks sampled
during the timed region, the add-min issue rate measured live, a structure
check (an Erdos-Renyi graph of the same n), the n = 16384 variants (general
path, fp32 with its own roofline, min-plus product, repeated squaring), the
serving replay (p50/p99 latency and solves/s against one-at-a-time solves)
and the CPU-oracle baseline.

  python bench.py [--gpus N --steps K --warmup W] [--workload roll64k]
  python bench.py --impl reference ...   # the CPU oracle timed as the reference arm

Multi-GPU (torchrun, N > 1): every rank solves its own replica of the workload
(the solve is not sharded), timing is max over ranks, value = all ranks'
relaxations / that time ("weak" scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "APSP GRelax/s (n³/s) int32 vs packed-int16; serving p50/p99 ms and solves/s"
UNIT = "GRelax/s"
ADDMIN_LANES_PER_CLK_PER_SM = 64  # add-min lane-ops per clock per SM: 64 INT32 lanes per SM, as apsp_addmin_peak measures
WORKLOAD_TEXT = {
    "gmm16k": "n=16384 symmetric k=10 kNN graph over a 10-D 8-component Gaussian mixture (seed 1), "
              "int32 weights max(1, rint(50 d)), dense INF-padded adjacency matrix",
    "roll64k": "n=65536 symmetric k=10 kNN Swiss-roll graph (seed 2), int32 weights max(1, rint(4 d))",
    "roll512": "n=512 symmetric k=8 kNN Swiss-roll graph (seed 0), int32 weights max(1, rint(100 d))",
    "er8k": "n=8192 Erdos-Renyi graph, average degree 16 plus a spanning path (seed 8), int32 weights U{1..1000}",
    "er16k": "n=16384 Erdos-Renyi graph, average degree 16 plus a spanning path (seed 16), int32 weights U{1..1000}",
    "er4k": "n=4096 Erdos-Renyi graph, average degree 16 plus a spanning path (seed 4), int32 weights U{1..1000}",
    "er32k": "n=32768 Erdos-Renyi graph, average degree 16 plus a spanning path (seed 32), int32 weights U{1..1000}",
    "er64k": "n=65536 Erdos-Renyi graph, average degree 16 plus a spanning path (seed 64), int32 weights U{1..1000}",
}
PAPER_CONTEXT = {
    "source": "paper Table 3 (Blocked-CB, Spark, 64 Xeon Gold 6130 cores, n=16384 Erdos-Renyi): 2m50s",
    "gops": 25.9,
}


# ----------------------------------------------------------------------------- helpers
def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1902_04446_gb300", "csrc")
    for f in ("fw_kernels.cu", "fw_device.cuh", "fw_tasks.cuh", "tma.cuh", "fw_launch.h"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch from a committed ncu summary, when it matches the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    cur = source_hash()
    for line in open(p):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel_key and parts[1] == cur:
            return float(parts[2])
    return None


def load_graph(name):
    if name.startswith("er"):
        n = {"er4k": 4096, "er8k": 8192, "er16k": 16384, "er32k": 32768, "er64k": 65536}[name]
        s, d, w = gen.er_graph(n, n // 1024)
        return gen.graphs.Graph(name, n, s, d, w, "int32")
    return gen.workload(name)


def load_workload(name):
    g = load_graph(name)
    W = gen.dense_matrix(g.n, g.src, g.dst, g.w, dtype=np.int32)
    return g, W


def dense_on_device(torch, g, dtype, inf, device):
    """The dense adjacency matrix built on the device from the edge list (same
    convention as gen.dense_matrix: 0 diagonal, INF for non-edges, min over
    duplicates)."""
    n = g.n
    W = torch.full((n, n), inf, dtype=dtype, device=device)
    src = torch.from_numpy(np.concatenate([g.src, g.dst]).astype(np.int64)).to(device)
    dst = torch.from_numpy(np.concatenate([g.dst, g.src]).astype(np.int64)).to(device)
    w = torch.from_numpy(np.concatenate([g.w, g.w])).to(device=device, dtype=dtype)
    W.view(-1).scatter_reduce_(0, src * n + dst, w, reduce="amin")
    W.fill_diagonal_(0)
    return W


# ----------------------------------------------------------------------------- GPU arm
def timed_solves(torch, h, dtype, Wd, Dd, steps, warmup, dist=None, profile=False):
    """Warm-up solves, then exactly `steps` solves bracketed by barrier + sync; returns (ms, launches, prof)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        h.solve_t(dtype, Wd, Dd)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if profile:
        h.profile(True)
        h.profile_read()
    l0 = h.launch_count
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        h.solve_t(dtype, Wd, Dd)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = h.launch_count - l0
    prof = h.profile_read() if profile else None
    if profile:
        h.profile(False)
    if h.last_status() != 0:
        raise RuntimeError(f"input check failed during the {dtype} benchmark")
    return ms, launches, prof


def _reduce_device(dist):
    # NCCL reduces CUDA tensors; gloo (CPU tests of the multi-rank logic) CPU tensors
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(torch, dist, x):
    """Timing across ranks: the slowest rank's time."""
    if dist is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(torch, dist, x):
    """Work across ranks: every rank solves its own replica, the job did the sum."""
    if dist is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_value(torch, dist, relax_per_rank, ms_this_rank):
    """Whole-job GRelax/s: all ranks' relaxations / the slowest rank's time."""
    ms = max_over_ranks(torch, dist, ms_this_rank)
    return sum_over_ranks(torch, dist, relax_per_rank) / (ms / 1e3) / 1e9, ms


def sample_graph(workload: str, n_s: int):
    """The workload's generator recipe at a smaller vertex count (for the CPU oracle)."""
    if workload.startswith("gmm"):
        s, d, dist = gen.knn_edges(gen.gaussian_mixture(n_s, 1), 10)
        return s, d, gen.int_weights(dist, 50.0)
    if workload.startswith("roll"):
        k, scale, seed = {"roll512": (8, 100.0, 0), "roll64k": (10, 4.0, 2)}.get(workload, (10, 4.0, 2))
        s, d, dist = gen.knn_edges(gen.swiss_roll(n_s, seed), k)
        return s, d, gen.int_weights(dist, scale)
    return gen.er_graph(n_s, 8)


def oracle_full_fw(workload: str, n_s: int):
    """Times the oracle's complete Floyd-Warshall on the workload's recipe at n_s vertices.

    A complete run is the honest sample: a slice of early outer iterations
    would be much faster than the whole (the oracle skips rows whose d(i,k) is
    still INF, and early in the run most are).
    """
    import oracle
    s, d, w = sample_graph(workload, n_s)
    W = gen.dense_matrix(n_s, s, d, w, dtype=np.int64)
    t0 = time.perf_counter()
    oracle.fw(W)
    return time.perf_counter() - t0


def cpu_baseline(workload: str, n_s: int = 4096, n_full: int | None = None):
    """The oracle (single-threaded C Floyd-Warshall), complete run on a bounded sample of the workload, with the
    n^3 extrapolation of its time to the workload's own n (labelled as such: a full run there takes days)."""
    dt = oracle_full_fw(workload, n_s)
    rate = float(n_s) ** 3 / dt / 1e9
    out = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"the oracle's complete int64 Floyd-Warshall on the same generator recipe at n={n_s} "
                     f"({dt:.1f} s on one host core); value = n^3 / t"}
    if n_full and n_full > n_s:
        out["extrapolated"] = {"n": n_full, "seconds": float(n_full) ** 3 / (rate * 1e9),
                               "how": "n^3 extrapolation of the measured rate (not measured)"}
    return out


def _replay_batched(torch, apsp, device, mats, arrival, **cfg):
    """Submits request i at arrival[i] (seconds from start) and polls to completion."""
    nreq = len(mats)
    with apsp.Handle(device=device, **cfg) as h:
        for W in mats[:8]:  # warm-up
            t = h.submit(W)
            h.wait(t)
            h.release(t)
        lat = [None] * nreq
        tickets, pending = {}, set()
        t_start = time.perf_counter()
        i = 0
        while i < nreq or pending:
            now = time.perf_counter() - t_start
            while i < nreq and arrival[i] <= now:
                tickets[i] = h.submit(mats[i])
                pending.add(i)
                i += 1
            done = []
            for j in pending:
                st, _, rc = h.poll(tickets[j])
                if st == 3:
                    lat[j] = (time.perf_counter() - t_start) - arrival[j]
                    done.append(j)
                elif st == 4:
                    raise RuntimeError(f"serving request {j} failed with status {rc}")
            for j in done:
                pending.discard(j)
                h.release(tickets[j])
            if not done and (i >= nreq or arrival[i] > now + 1e-4):
                time.sleep(1e-5)
        return lat, time.perf_counter() - t_start


def _replay_single(torch, apsp, device, mats, arrival):
    """FIFO one-at-a-time apsp_solve calls, each synchronized, starting no earlier than its arrival."""
    nreq = len(mats)
    with apsp.Handle(device=device) as h:
        for W in mats[:8]:
            h.solve_t("int32", W)
        torch.cuda.synchronize()
        lat = []
        t_start = time.perf_counter()
        for j in range(nreq):
            now = time.perf_counter() - t_start
            if arrival[j] > now:
                time.sleep(arrival[j] - now)
            h.solve_t("int32", mats[j])
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - t_start) - arrival[j])
        return lat, time.perf_counter() - t_start


def serving_replay(torch, apsp, device, nreq, **cfg):
    """The Poisson trace through the request loop (continuous batching into the
    batched persistent kernel) and through one-at-a-time solves; then the same
    requests all submitted at once (saturation throughput)."""
    arrival, ns, seeds = gen.serving_trace(num=nreq)
    mats = []
    for s in seeds:
        r = gen.graphs.serving_request(int(s))
        n = r.n
        W = torch.full((n, n), apsp.INF_I32, dtype=torch.int32, device=device)
        src = torch.from_numpy(np.concatenate([r.src, r.dst])).to(device)
        dst = torch.from_numpy(np.concatenate([r.dst, r.src])).to(device)
        w = torch.from_numpy(np.concatenate([r.w, r.w]).astype(np.int32)).to(device)
        W.view(-1).scatter_reduce_(0, src * n + dst, w, reduce="amin")
        W.fill_diagonal_(0)
        mats.append(W)
    torch.cuda.synchronize()
    relax = float(np.sum(ns.astype(np.float64) ** 3))

    def summary(lat, span):
        lat = np.asarray(lat)
        return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "solves_per_s": nreq / span, "grelax_per_s": relax / span / 1e9}

    out = {"requests": nreq, "offered_req_per_s": 200.0,
           "n": "log-uniform [128, 4096], ER avg degree 16 + spanning path, int32 weights U{1..1000}",
           "inputs": "adjacency matrices resident on the device at arrival"}
    out["batched"] = summary(*_replay_batched(torch, apsp, device, mats, arrival, **cfg))
    out["one_at_a_time"] = summary(*_replay_single(torch, apsp, device, mats, arrival))
    zero = np.zeros_like(arrival)
    sat_b = summary(*_replay_batched(torch, apsp, device, mats, zero, **cfg))
    sat_s = summary(*_replay_single(torch, apsp, device, mats, zero))
    out["saturated"] = {"batched_solves_per_s": sat_b["solves_per_s"], "one_at_a_time_solves_per_s":
                        sat_s["solves_per_s"], "batched_grelax_per_s": sat_b["grelax_per_s"],
                        "one_at_a_time_grelax_per_s": sat_s["grelax_per_s"],
                        "note": "all requests submitted at t=0"}
    # the batched persistent kernel by itself: the trace's requests below 1536 vertices in launches of 64
    small = [i for i in range(nreq) if mats[i].shape[0] < 1536]
    with apsp.Handle(device=device) as h:
        outs = [torch.empty_like(mats[i]) for i in small]
        h.solve_batch([mats[i] for i in small[:64]], outs[:64])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(0, len(small), 64):
            h.solve_batch([mats[i] for i in small[k:k + 64]], outs[k:k + 64])
        e1.record()
        torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    props = torch.cuda.get_device_properties(device)
    peak = ADDMIN_LANES_PER_CLK_PER_SM * props.multi_processor_count * 2070e6
    # relaxations the kernel performs: every round of every graph updates its whole tile grid (128 x 128 tiles,
    # round width 64, general mode)
    done = 0.0
    for i in small:
        n = mats[i].shape[0]
        tiles = -(-n // 128)
        done += (-(-n // 64)) * (tiles * 128) ** 2 * 64
    out["batched_kernel"] = {"graphs": len(small), "launches": -(-len(small) // 64), "seconds": sec,
                             "grelax_per_s_n3": float(np.sum(np.array([mats[i].shape[0] for i in small],
                                                                      dtype=np.float64) ** 3)) / sec / 1e9,
                             "grelax_per_s_performed": done / sec / 1e9, "frac_of_addmin_peak": done / sec / peak,
                             "note": "the trace's requests with n < 1536 in batched launches of 64; performed = "
                                     "whole 128 x 128 tiles, every round"}
    return out


def addmin_peaks(apsp, device):
    """The add-min issue rate of each dtype's add-min form, measured live on this GPU (apsp_addmin_peak)."""
    import ctypes
    L = apsp.get_lib()
    out = {}
    for name, code in (("int32", apsp.APSP_I32), ("u16x2", apsp.APSP_U16), ("fp32", apsp.APSP_F32)):
        rpc, rps = ctypes.c_double(), ctypes.c_double()
        if L.apsp_addmin_peak(device, code, ctypes.byref(rpc), ctypes.byref(rps)) == 0:
            out[name] = {"relax_per_clk_per_sm": rpc.value, "grelax_per_s_event_timed": rps.value / 1e9}
    return out


def phase3_rate(prof):
    """Relaxations per second of the Phase-3 launches (the dominant kernel), from the per-launch CUDA events."""
    n3, ms3, r3 = prof[3]
    return (r3 / (ms3 / 1e3) / 1e9) if n3 and ms3 else None


def e2e_measure(torch, h, Wd, Dd, steps, warmup, dist):
    """End to end through the public API with host buffers (pinned), copies inside the timed region: every step
    copies its input in and its result out; one copy stream moves step i+1's input in and another step i-1's
    result out while step i solves (two device buffer pairs), so the copy engines work beside the solve."""
    device = Wd.device
    Wh = torch.empty(Wd.shape, dtype=Wd.dtype, pin_memory=True)
    Wh.copy_(Wd)
    Dh = torch.empty(Wd.shape, dtype=Wd.dtype, pin_memory=True)
    stream = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(device), torch.cuda.Stream(device)
    Wb, Db = [Wd, torch.empty_like(Wd)], [Dd, torch.empty_like(Dd)]

    def run(k):
        solved = [None, None]  # per buffer pair: the event after its last solve
        out_done = [None, None]  # per buffer pair: the event after its last copy out
        for i in range(k):
            b = i & 1
            with torch.cuda.stream(s_in):
                if solved[b] is not None:
                    s_in.wait_event(solved[b])  # the solve two steps back has read this input buffer
                Wb[b].copy_(Wh, non_blocking=True)
                ev_in = torch.cuda.Event()
                ev_in.record(s_in)
            stream.wait_event(ev_in)
            if out_done[b] is not None:
                stream.wait_event(out_done[b])  # the result two steps back has left this buffer
            h.solve_t("int32", Wb[b], Db[b])
            solved[b] = torch.cuda.Event()
            solved[b].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(solved[b])
                Dh.copy_(Db[b], non_blocking=True)
                out_done[b] = torch.cuda.Event()
                out_done[b].record(s_out)

    run(max(1, warmup))
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run(steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist is not None:
        dist.barrier()
    # the last result on the host equals the device result (rows sampled: the matrix can be 17 GB)
    last = Db[(steps - 1) & 1]
    rows = torch.linspace(0, Wd.shape[0] - 1, 64, dtype=torch.long)
    if not torch.equal(Dh[rows], last[rows.to(last.device)].cpu()):
        raise RuntimeError("end-to-end result on the host differs from the device result")
    nbytes = int(Wh.numel() * Wh.element_size())
    del Wb, Db, Wh, Dh
    return wall * 1e3, nbytes


def serving_breakdown(torch, apsp, device, nreq=2000):
    """Where the serving trace's GPU time goes (one JSON line, not the contract line): its matrices solved back to
    back on one stream (all, the n >= 1536 ones, the smaller ones), the smaller ones in batched launches of 64,
    and all of them spread over four streams."""
    arrival, ns, seeds = gen.serving_trace(num=nreq)
    mats = []
    for sd in seeds:
        r = gen.graphs.serving_request(int(sd))
        mats.append(dense_on_device(torch, gen.graphs.Graph("req", r.n, r.src, r.dst, r.w, "int32"), torch.int32,
                                    apsp.INF_I32, device))
    outs = [torch.empty_like(W) for W in mats]
    ns = np.array([W.shape[0] for W in mats])
    big = [i for i in range(nreq) if ns[i] >= 1536]
    small = [i for i in range(nreq) if ns[i] < 1536]
    res = {"requests": nreq, "n_ge_1536": len(big), "n_lt_1536": len(small),
           "relax_share_n_ge_1536": float(np.sum(ns[big].astype(float) ** 3) / np.sum(ns.astype(float) ** 3))}

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    with apsp.Handle(device=device) as h:
        for i in range(20):
            h.solve_t("int32", mats[i], outs[i])
        res["one_stream_all_s"] = timed(lambda: [h.solve_t("int32", mats[i], outs[i]) for i in range(nreq)])
        res["one_stream_n_ge_1536_s"] = timed(lambda: [h.solve_t("int32", mats[i], outs[i]) for i in big])
        res["one_stream_n_lt_1536_s"] = timed(lambda: [h.solve_t("int32", mats[i], outs[i]) for i in small])
        res["batched_64_n_lt_1536_s"] = timed(
            lambda: [h.solve_batch([mats[i] for i in small[k:k + 64]], [outs[i] for i in small[k:k + 64]])
                     for k in range(0, len(small), 64)])
    hs = [apsp.Handle(device=device) for _ in range(4)]
    sts = [torch.cuda.Stream(device) for _ in range(4)]
    t0 = time.perf_counter()
    for i in range(nreq):
        hs[i % 4].solve_t("int32", mats[i], outs[i], stream=sts[i % 4])
    torch.cuda.synchronize()
    res["four_streams_all_s"] = time.perf_counter() - t0
    for h in hs:
        h.close()
    print(json.dumps({"serving_breakdown": res}), flush=True)


def run_gpu(args):
    import torch

    import paper_1902_04446_gb300 as apsp

    ws, rank, local = dist_info()
    dist = None
    if ws > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    device = local
    torch.cuda.set_device(device)
    props = torch.cuda.get_device_properties(device)
    sms = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    live = addmin_peaks(apsp, device)
    peak = ADDMIN_LANES_PER_CLK_PER_SM * sms * sm_max_mhz * 1e6 / 1e9  # GRelax/s, int32 (u16x2: twice)

    g = load_graph(args.workload)
    n = g.n
    Wd = dense_on_device(torch, g, torch.int32, 1073741823, device)
    Dd = torch.empty_like(Wd)
    h = apsp.Handle(device=device)
    relax_step = float(n) ** 3

    # ---- the headline: int32 solves of the workload, inputs resident in HBM
    with ClockSampler(device) as clk:
        ms, launches, prof = timed_solves(torch, h, "int32", Wd, Dd, args.steps, args.warmup, dist, profile=True)
    clocks = clk.summary()
    value, ms_max = job_value(torch, dist, relax_step * args.steps, ms)

    # roofline of the dominant kernel (Phase 3), from the live event timings
    achieved = phase3_rate(prof)
    phase_ms = {f"phase{p}": round(prof[p][1] / args.steps, 3) for p in (1, 2, 3)}
    if h.tuned_config("int32", n)[1] == 4:
        kname, kkey = ("fw_solve_ws<int32> (every round in one launch: Phase-3 tiles with each round's Phase 1 and "
                       "Phase 2 as tasks)"), "fw_solve_ws"
        work = ("relaxations performed in the launch: Phase 3 (in symmetric mode only the tiles touching the upper "
                "triangle) plus every round's Phase 1 and Phase 2")
    else:
        kname, kkey = "fw_phase3_ws<int32> (warp-specialized Phase 3, one launch per round)", "fw_phase3_ws"
        work = ("relaxations performed by the Phase-3 launches (in symmetric mode only the tiles touching the upper "
                "triangle)")
    roofline = {"bound": "alu", "kernel": kname,
                "achieved": achieved, "peak": peak, "unit": UNIT, "work": work,
                "frac": (achieved / peak) if achieved else None,
                "peak_basis": f"{ADDMIN_LANES_PER_CLK_PER_SM} add-min lanes/clk/SM (the SM's INT32 lanes; measured "
                              f"live: {live.get('int32', {}).get('relax_per_clk_per_sm', float('nan')):.1f}) x "
                              f"{sms} SMs x {sm_max_mhz:.0f} MHz (max SM clock)",
                "traffic": ncu_traffic(f"{kkey}_int32_{args.workload}"),
                "traffic_unit": "DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "phase_ms_per_step": phase_ms,
                "phase3_launches_per_step": prof[3][0] // max(1, args.steps),
                "phase3_share_of_step": prof[3][1] / ms if ms else None}
    if clocks and achieved:
        roofline["frac_at_median_clock"] = achieved / (ADDMIN_LANES_PER_CLK_PER_SM * sms * clocks["sm_mhz"] / 1e3)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "int32", "data": "synthetic",
           "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT.get(args.workload, '')}", "n": n,
                      "edges": int(g.src.shape[0]), "round_width": h.tuned_config("int32", n)[0],
                      "parallelism": f"replicas x{ws}",
                      "l2": "input matrix larger than L2 (%.2f GB), no flush needed" % (n * n * 4 / 1e9)},
           "roofline": roofline, "gpu_launches": int(launches), "clocks": clocks,
           "addmin_peak_live": live, "paper_context": PAPER_CONTEXT}

    # ---- the packed 16-bit half of the metric, on the same graph and the same steps
    if not args.no_variants:
        ms16, l16, prof16 = timed_solves(torch, h, "auto", Wd, Dd, args.steps, args.warmup, dist, profile=True)
        v16, ms16 = job_value(torch, dist, relax_step * args.steps, ms16)
        a16 = phase3_rate(prof16)
        out["packed_u16"] = {"value": v16, "unit": UNIT, "ms_per_step": ms16 / args.steps,
                             "speedup_vs_int32": v16 / value, "path": "apsp_solve(APSP_AUTO): bound pass, pack, "
                             "u16x2 rounds, unpack (all inside the timed region)",
                             "phase3_achieved": a16, "phase3_peak": 2 * peak,
                             "phase3_frac": (a16 / (2 * peak)) if a16 else None, "gpu_launches": int(l16),
                             "round_width": h.tuned_config("u16", n)[0], "bytes_per_distance": 2}

    # ---- the same graph in upper-triangular storage (half the bytes): edge list -> storage -> rounds, fewer
    # repeats (each step rebuilds the matrix from the edge list, as the dense path's step copies W in)
    if not args.no_variants:
        reps = min(args.steps, 2)
        src = torch.from_numpy(g.src.astype(np.int32)).to(device)
        dst = torch.from_numpy(g.dst.astype(np.int32)).to(device)
        ww = torch.from_numpy(g.w.astype(np.int32)).to(device)
        rows_, ld_, tbytes = apsp.tri_layout("int32", n)
        T = apsp.tri_empty("int32", n, device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(1):
            h.tri_from_edges("int32", src, dst, ww, n, T)
            h.solve_tri("int32", T, n)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            h.tri_from_edges("int32", src, dst, ww, n, T)
            h.solve_tri("int32", T, n)
        e1.record()
        torch.cuda.synchronize()
        if h.last_status() != 0:
            raise RuntimeError("upper-triangular solve: input check or bounded wait failed")
        mst = e0.elapsed_time(e1)
        pick = torch.linspace(0, n - 1, 16, dtype=torch.long, device=Dd.device)
        if not torch.equal(apsp.tri_rows("int32", T, n, pick), Dd[pick]):
            raise RuntimeError("upper-triangular result differs from the dense solve")
        vt, mst = job_value(torch, dist, relax_step * reps, mst)
        out["upper_triangular_int32"] = {
            "value": vt, "unit": UNIT, "ms_per_step": mst / reps, "repeats": reps,
            "storage_bytes": tbytes, "dense_storage_bytes": n * n * 4, "storage_ratio": tbytes / (n * n * 4),
            "path": "apsp_tri_from_edges + apsp_solve_tri: only the super-tiles (I <= J) stored, folded into one "
                    "rectangle; rows checked against the dense solve"}
        del T, src, dst, ww
        torch.cuda.empty_cache()

    # ---- end to end through host buffers, same graph and steps
    mse, nbytes = e2e_measure(torch, h, Wd, Dd, args.steps, args.warmup, dist)
    mse = max_over_ranks(torch, dist, mse)
    out["e2e"] = {"value": sum_over_ranks(torch, dist, relax_step * args.steps) / (mse / 1e3) / 1e9, "unit": UNIT,
                  "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                  "ms_per_step": mse / args.steps,
                  "pipeline": "pinned host buffers; step i+1's copy in and step i-1's copy out overlap step i's "
                              "solve (two copy streams, two device buffer pairs); host wall clock from the first "
                              "copy in to the last copy out"}
    torch.cuda.empty_cache()

    if not args.no_variants:
        # structure-obliviousness (the paper's Sec. 5.1: runtime depends only on n): the same solve on an
        # Erdos-Renyi graph with the same n; fewer repeats at the large sizes
        er_name = {16384: "er16k", 65536: "er64k"}.get(n)
        if er_name and not args.workload.startswith("er"):
            reps = args.steps if n <= 16384 else min(args.steps, 2)
            ge = load_graph(er_name)
            We = dense_on_device(torch, ge, torch.int32, 1073741823, device)
            mse_er, _, _ = timed_solves(torch, h, "int32", We, Dd, reps, 1, dist)
            ms_w, _, _ = timed_solves(torch, h, "int32", Wd, Dd, reps, 0, dist)
            out["structure_check"] = {"er_ms_per_step": mse_er / reps, "workload_ms_per_step": ms_w / reps,
                                      "ratio": (mse_er / reps) / (ms_w / reps), "graph": WORKLOAD_TEXT[er_name],
                                      "repeats": reps}
            del We
        del Wd, Dd
        torch.cuda.empty_cache()
        out.update(extras_gmm16k(torch, apsp, h, args, dist, device, peak, live, sms, sm_max_mhz))
    else:
        del Wd, Dd
    h.close()

    if rank == 0 and not args.no_serving:
        out["serving"] = serving_replay(torch, apsp, device, args.serving_requests)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, n_full=n)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def extras_gmm16k(torch, apsp, h, args, dist, device, peak, live, sms, sm_max_mhz):
    """The other variants, on the n = 16384 workload (one solve takes ~0.1 s there): the general (non-symmetric)
    path, fp32 weights with their own Phase-3 roofline, the min-plus product and repeated squaring."""
    out = {}
    g = load_graph("gmm16k")
    n = g.n
    relax_step = float(n) ** 3
    W = dense_on_device(torch, g, torch.int32, 1073741823, device)
    D = torch.empty_like(W)
    with apsp.Handle(device=device, symmetric=2) as hg:
        msg, lg, profg = timed_solves(torch, hg, "int32", W, D, args.steps, args.warmup, dist, profile=True)
    vg, msg = job_value(torch, dist, relax_step * args.steps, msg)
    ag = phase3_rate(profg)
    out["general_int32"] = {"workload": "gmm16k: " + WORKLOAD_TEXT["gmm16k"], "value": vg, "unit": UNIT,
                            "ms_per_step": msg / args.steps,
                            "path": "symmetric mode off: every Phase-3 tile updated, no mirror pass",
                            "phase3_achieved": ag, "phase3_frac": (ag / peak) if ag else None,
                            "gpu_launches": int(lg)}
    del W, D
    gf = gen.workload("gmm16k_f32")
    gf = gen.graphs.Graph(gf.name, gf.n, gf.src, gf.dst, gf.w.astype(np.float32), "fp32")
    Wf = dense_on_device(torch, gf, torch.float32, float("inf"), device)
    Df = torch.empty_like(Wf)
    msf, lf, proff = timed_solves(torch, h, "fp32", Wf, Df, args.steps, args.warmup, dist, profile=True)
    vf, msf = job_value(torch, dist, relax_step * args.steps, msf)
    af = phase3_rate(proff)
    f_rpc = live.get("fp32", {}).get("relax_per_clk_per_sm")
    peak_f = f_rpc * sms * sm_max_mhz / 1e3 if f_rpc else None
    kf = "fw_solve_ws<fp32> (every round in one launch)" if h.tuned_config("fp32", n)[1] == 4 else \
        "fw_phase3_ws<fp32> (one launch per round)"
    out["fp32"] = {"workload": "gmm16k_f32: the gmm16k points, raw Euclidean distances as fp32 weights",
                   "value": vf, "unit": UNIT, "ms_per_step": msf / args.steps, "gpu_launches": int(lf),
                   "roofline": {"bound": "alu", "kernel": kf, "achieved": af, "peak": peak_f, "unit": UNIT,
                                "frac": (af / peak_f) if (af and peak_f) else None,
                                "peak_basis": f"relaxations/clk/SM of the fp32 tile's instruction form (packed pair "
                                              f"add + three-input min) measured live ({f_rpc:.1f}) x {sms} SMs x "
                                              f"{sm_max_mhz:.0f} MHz" if f_rpc else None,
                                "frac_of_int32_peak": (af / peak) if af else None}}
    del Wf, Df

    # the min-plus product as a library primitive (Table 1 MatProd + MatMin)
    # and repeated squaring (Alg. 1) as a second workload
    mk = 8192
    gmp = torch.Generator(device="cuda").manual_seed(8192)
    A = torch.randint(0, 1000, (mk, mk), dtype=torch.int32, device="cuda", generator=gmp)
    B = torch.randint(0, 1000, (mk, mk), dtype=torch.int32, device="cuda", generator=gmp)
    C = torch.full((mk, mk), 1073741823, dtype=torch.int32, device="cuda")
    for _ in range(max(1, args.warmup)):
        h.minplus(A, B, C)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        h.minplus(A, B, C)
    e1.record()
    torch.cuda.synchronize()
    msmp = e0.elapsed_time(e1) / args.steps
    gr = float(mk) ** 3 / (msmp / 1e3) / 1e9
    out["minplus"] = {"m": mk, "k": mk, "n": mk, "dtype": "int32", "ms": msmp, "value": gr, "unit": UNIT,
                      "frac_of_addmin_peak": gr / peak, "inputs": "uniform U{0..999} (torch generator seed 8192)"}
    del A, B, C
    gs = load_graph("er4k")
    Ws = dense_on_device(torch, gs, torch.int32, 1073741823, device)
    Ds = torch.empty_like(Ws)
    h.solve_squaring("int32", Ws, Ds)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        h.solve_squaring("int32", Ws, Ds)
    e1.record()
    torch.cuda.synchronize()
    mss = e0.elapsed_time(e1) / args.steps
    msfw, _, _ = timed_solves(torch, h, "int32", Ws, Ds, args.steps, 1, None)
    nsq = gs.n
    prods = int(np.ceil(np.log2(nsq - 1)))
    out["squaring"] = {"graph": WORKLOAD_TEXT["er4k"], "n": nsq, "products": prods,
                       "ms_per_solve": mss, "products_grelax_per_s": prods * float(nsq) ** 3 / (mss / 1e3) / 1e9,
                       "floyd_warshall_ms_per_solve": msfw / args.steps,
                       "path": "apsp_solve_squaring (Alg. 1): ceil(log2(n-1)) in-place min-plus products"}
    del Ws, Ds
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, n_s: int = 2048):
    """The CPU oracle as the reference arm: each step is its complete Floyd-Warshall on a bounded sample."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_full_fw(args.workload, n_s)
    times = [oracle_full_fw(args.workload, n_s) for _ in range(args.steps)]
    dt = sum(times)
    value = args.steps * float(n_s) ** 3 / dt / 1e9
    sample = (f"each step = the oracle's complete int64 Floyd-Warshall on the workload's generator recipe at "
              f"n={n_s} (one host core); value = n^3 / t")
    n = {"gmm16k": 16384, "er4k": 4096, "er8k": 8192, "er16k": 16384, "roll64k": 65536,
         "roll512": 512}.get(args.workload)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT.get(args.workload, '')}", "n": n,
                      "sample_n": n_s},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_cpu_sweep(args):
    """The oracle's single-threaded Floyd-Warshall timed on the host at several n (one JSON line, not the contract
    line), with an n^3 extrapolation to the full sizes from the largest measured n, the paper's single-core
    reference (T_1 = 0.022 s at n = 256, SciPy's Floyd-Warshall, Sec. 5.4) beside it, and the multi-threaded
    Dijkstra verifier's time per source row (verification, not a baseline)."""
    import platform

    import oracle
    sizes = tuple(int(x) for x in args.cpu_sweep_sizes.split(","))
    rows = []
    for n_s in sizes:
        reps = 5 if n_s <= 512 else 1
        dt = min(oracle_full_fw(args.workload, n_s) for _ in range(reps))
        rows.append({"n": n_s, "seconds": dt, "grelax_per_s": float(n_s) ** 3 / dt / 1e9})
    rate = rows[-1]["grelax_per_s"]
    extrap = {str(n): {"seconds_extrapolated": float(n) ** 3 / (rate * 1e9)} for n in (16384, 65536, 262144)}
    g = load_graph("gmm16k")
    threads = max(1, min(os.cpu_count() or 1, 64))
    src = np.arange(0, g.n, 32)
    t0 = time.perf_counter()
    oracle.dijkstra(g.n, g.src, g.dst, g.w, src, threads=threads)
    dv = time.perf_counter() - t0
    print(json.dumps({"cpu_sweep": "oracle int64 Floyd-Warshall, one host core", "workload_recipe": args.workload,
                      "host": {"machine": platform.machine(), "processor": platform.processor(),
                               "cpu_count": os.cpu_count()},
                      "measured": rows, "extrapolated_n3": extrap,
                      "paper_single_core": {"n": 256, "seconds": 0.022, "grelax_per_s": 256 ** 3 / 0.022 / 1e9,
                                            "source": "Sec. 5.4, SciPy Floyd-Warshall on one core"},
                      "verifier": {"what": "oracle Dijkstra rows on gmm16k (verification, not a baseline)",
                                   "rows": int(src.shape[0]), "threads": threads, "seconds": dv,
                                   "ms_per_row_per_thread": dv / src.shape[0] * threads * 1e3}}), flush=True)


def run_round_shapes(args):
    """Round shapes (round width x Phase-3 kernel) on the workload in one dtype, one JSON line each (not the
    contract line): the table the autotuner chooses from and the default by n comes from, with per-phase times."""
    import torch

    import paper_1902_04446_gb300 as apsp

    if args.er_n:
        s_, d_, w_ = gen.er_graph(args.er_n, args.er_n)
        g = gen.graphs.Graph(f"er n={args.er_n}", args.er_n, s_, d_, w_, "int32")
    else:
        g = load_graph(args.workload)
    n = g.n
    Wd = dense_on_device(torch, g, torch.int32, 1073741823, 0)
    if args.dtype == "u16":
        Wd = torch.where(Wd >= 1073741823, torch.full_like(Wd, 0x7FFF), Wd).to(torch.int16)
    elif args.dtype == "fp32":
        Wd = torch.where(Wd >= 1073741823, torch.full(Wd.shape, float("inf"), device=Wd.device), Wd.float())
    Dd = torch.empty_like(Wd)
    names = {1: "one CTA per tile", 2: "TMA, 256 threads", 3: "TMA, 512 threads",
             4: "warp-specialized, one launch per round", 5: "warp-specialized, every round in one launch"}
    epw = 2 if args.dtype == "u16" else 1
    peak = ADDMIN_LANES_PER_CLK_PER_SM * torch.cuda.get_device_properties(0).multi_processor_count * 2070.0 / 1e3
    shapes = [(bk, v) for bk in (32, 64) for v in (1, 2, 3, 4, 5)] + [(128, 1), (128, 4)]
    if args.shapes:
        shapes = [tuple(int(x) for x in sv.split("x")) for sv in args.shapes.split(",")]
    for bk, v in shapes:
        with apsp.Handle(device=0, block_k=bk, phase3_variant=v) as h:
            # the solve time without per-phase events (they cost the per-round launches time), then the phases
            ms, launches, _ = timed_solves(torch, h, args.dtype, Wd, Dd, args.steps, args.warmup, None)
            _, _, prof = timed_solves(torch, h, args.dtype, Wd, Dd, args.steps, 0, None, profile=True)
            status = h.last_status()
        ms /= args.steps
        n3, ms3, r3 = prof[3]
        print(json.dumps({"workload": g.name if args.er_n else args.workload, "n": n, "dtype": args.dtype,
                          "round_width": bk, "phase3_variant": v,
                          "phase3_kernel": names[v], "ms_per_solve": round(ms, 2),
                          "grelax_per_s": float(n) ** 3 / (ms / 1e3) / 1e9,
                          "phase_ms": {f"phase{p}": round(prof[p][1] / args.steps, 2) for p in (1, 2, 3)},
                          "phase3_frac_of_addmin_peak_2070mhz":
                              (r3 / (ms3 / 1e3) / 1e9 / (peak * epw)) if ms3 else None,
                          "launches_per_solve": launches // args.steps, "status": status}), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="roll64k", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--round-shapes", action="store_true",
                    help="time every round shape (round width x Phase-3 kernel) instead of the benchmark line")
    ap.add_argument("--dtype", default="int32", choices=["int32", "u16", "fp32"],
                    help="--round-shapes: the element type solved (u16 from the int32 matrix, INF -> 0x7FFF)")
    ap.add_argument("--shapes", default="",
                    help="--round-shapes: comma-separated BKxVARIANT list (e.g. 64x4,64x5); default all twelve (width "
                         "128 runs variants 1 and 4)")
    ap.add_argument("--er-n", type=int, default=0,
                    help="--round-shapes: an Erdos-Renyi graph of this n (average degree 16 plus a spanning path, "
                         "seed n, weights U{1..1000}) instead of --workload")
    ap.add_argument("--cpu-sweep", action="store_true",
                    help="time the CPU oracle at several n (and the Dijkstra verifier) instead of the benchmark line")
    ap.add_argument("--cpu-sweep-sizes", default="256,512,1024,2048,4096",
                    help="--cpu-sweep: comma-separated n to time the oracle at (16384 takes about 6 minutes)")
    ap.add_argument("--addmin-peak", action="store_true",
                    help="print the add-min issue rate of each dtype measured on this GPU (apsp_addmin_peak) and exit")
    ap.add_argument("--serving-breakdown", action="store_true",
                    help="print where the serving trace's GPU time goes (solves back to back, batched, four streams)")
    args = ap.parse_args(argv)
    if args.serving_breakdown:
        import torch

        import paper_1902_04446_gb300 as apsp
        serving_breakdown(torch, apsp, 0, args.serving_requests)
    elif args.addmin_peak:
        import torch

        import paper_1902_04446_gb300 as apsp
        p = torch.cuda.get_device_properties(0)
        print(json.dumps({"gpu": p.name, "sms": p.multi_processor_count, "addmin_peak": addmin_peaks(apsp, 0)}),
              flush=True)
    elif args.cpu_sweep:
        run_cpu_sweep(args)
    elif args.round_shapes:
        run_round_shapes(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
