"""The stage hand-off of the warp-specialized Phase-3 kernel, as a model run on the host (no GPU).

`fw_phase3_ws` (csrc/fw_kernels.cu) moves data between one producer warp and 8 consumer warps through
mbarriers: full[s] / empty[s] for the two A/B stages, cdone and cfree for the C buffer (the min-reduction
epilogue of int32 and fp32; packed 16-bit uses full_c instead of cfree, not modelled here).  With round
width 128 a tile takes two stages in a row (NSPLIT = 2): the producer streams (tile, k-half) items, item j
in stage j & 1, waiting on empty[s] with parity (j >> 1) & 1, and the consumers wait on full[s] with the
same parity.  This model restates those rules -- which item goes to which stage, which parity every wait
uses, when each barrier is arrived on -- and runs the producer and the consumer warps in random orders.
It checks that every run completes, that every consumer reads the item it expects from each stage, that
the producer never refills a stage a consumer has not released, that each tile's C buffer is written only
after the previous tile's reduction has read it, and that no parity wait is ever two phases behind (an
mbarrier wait checks only the parity, so a waiter two phases behind would wrongly pass).
"""
import random

import pytest

NCW = 8  # consumer warps


class Bar:
    """An mbarrier: `count` arrivals complete a phase; completed = phases completed so far."""

    def __init__(self, count):
        self.count, self.pending, self.completed = count, count, 0

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0
        if self.pending == 0:
            self.completed += 1
            self.pending = self.count

    def ready(self, parity, k):
        """try_wait.parity for the k-th completion (0-based): true once that phase completed.  The hardware
        compares parities only; the model asserts that the waiter is never so far behind that the compare
        would give the wrong answer."""
        assert self.completed <= k + 1, "a waiter fell two phases behind: the parity compare would mislead it"
        assert parity == (k & 1)
        return self.completed >= k + 1


def run(n_tiles, nsplit, seed, mistake=None):
    """One random interleaving.  mistake (for the negative tests): "stage" -- a consumer takes the stage of
    the tile (i & 1) instead of the item's (j & 1); "refill" -- the producer refills a stage without waiting
    for its empty barrier; "cfree" -- the consumers write the C buffer without waiting for cfree."""
    rng = random.Random(seed)
    full = [Bar(1), Bar(1)]       # completed by the TMA (modelled: at issue)
    empty = [Bar(NCW), Bar(NCW)]  # one arrival per consumer warp
    cdone, cfree = Bar(NCW), Bar(1)
    stage = [None, None]          # the item a stage holds
    readers = [set(), set()]      # consumer warps that have not yet released the stage's current item
    cbuf = {"tile": None, "writers": set(), "read": True}
    n_items = n_tiles * nsplit
    log = []

    def producer():
        next_item = 0

        def issue(s):
            nonlocal next_item
            assert not readers[s], "stage refilled before every consumer released it"
            stage[s] = next_item
            readers[s] = set(range(NCW))
            full[s].arrive()
            next_item += 1

        issue(0)
        if n_items > 1:
            issue(1)
        for i in range(n_tiles):
            for h in range(nsplit):
                j = i * nsplit + h
                s = j & 1
                if mistake != "refill":
                    while not empty[s].ready((j >> 1) & 1, j >> 1):
                        yield
                else:
                    yield
                if j + 2 < n_items:
                    issue(s)
                    yield
            while not cdone.ready(i & 1, i):
                yield
            assert cbuf["tile"] == i and len(cbuf["writers"]) == NCW, "reduction of an incomplete C buffer"
            cbuf["read"] = True  # the reduction reads the buffer
            log.append(i)
            cfree.arrive()
            yield

    def consumer(w):
        for i in range(n_tiles):
            for h in range(nsplit):
                j = i * nsplit + h
                s = (i & 1) if mistake == "stage" else (j & 1)
                while not full[s].ready((j >> 1) & 1, j >> 1):
                    yield
                assert stage[s] == j, f"warp {w} read item {stage[s]} from stage {s}, expected {j}"
                yield  # the k-loop
                readers[s].discard(w)
                empty[s].arrive()
            yield  # the epilogue starts; the steps below are separate, as on the GPU
            if i > 0 and mistake != "cfree":
                while not cfree.ready((i - 1) & 1, i - 1):
                    yield
            if cbuf["tile"] != i:
                assert cbuf["read"], "C buffer overwritten before the previous reduction read it"
                cbuf.update(tile=i, writers=set(), read=False)
            cbuf["writers"].add(w)
            yield  # the stores and the proxy fence
            cdone.arrive()
            yield

    tasks = [producer()] + [consumer(w) for w in range(NCW)]
    live = list(range(len(tasks)))
    speed = [rng.choice((1, 2, 5, 20)) for _ in tasks]  # uneven speeds: warps drift apart as on the GPU
    steps = 0
    while live:
        k = rng.choices(live, weights=[speed[t] for t in live])[0]
        try:
            next(tasks[k])
        except StopIteration:
            live.remove(k)
        steps += 1
        assert steps < 200000, "no progress: a wait that never completes"
    assert log == list(range(n_tiles))
    return steps


@pytest.mark.parametrize("nsplit", [1, 2])
@pytest.mark.parametrize("n_tiles", [1, 2, 3, 5, 14])
def test_stage_handoff_completes_and_keeps_the_order(nsplit, n_tiles):
    for seed in range(40):
        assert run(n_tiles, nsplit, seed * 7919 + n_tiles) > n_tiles * nsplit


@pytest.mark.parametrize("mistake,nsplit", [("stage", 2), ("refill", 1), ("refill", 2), ("cfree", 1),
                                            ("cfree", 2)])
def test_the_model_catches_broken_rules(mistake, nsplit):
    """The model is not vacuous: with one rule broken, some interleaving fails a check."""
    failures = 0
    for seed in range(200):
        try:
            run(4, nsplit, seed, mistake)
        except AssertionError:
            failures += 1
    assert failures > 0
