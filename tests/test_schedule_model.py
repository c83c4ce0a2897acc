"""A model of the work-item schedule of the all-rounds Phase-3 kernel (fw_solve_ws), run on the CPU.

The kernel takes items from one device counter: block 0 holds round 0's Phase-1 and Phase-2 tasks, block j >= 1
round j-1's Phase-3 tiles (priority tiles first) with round j's tasks inserted; a tile waits for its round's tasks,
P1 of round j for round j-1's priority tiles and every tile of round j-2, the Phase-2 chunks for P1, the publication
for the chunks; 16-bit / fp32 tiles also for their previous round.  This model restates the item decode and those
rules in Python and drives G producer/consumer pairs under random interleavings, checking that every run completes,
that no rule is broken, and that every tile of every round and every task is processed exactly once.  It also shows
that a producer which blocks on a pending item (instead of queueing it and going on publishing its earlier tiles)
can stall -- the reason the kernel's producer never waits on another item.
"""
import random

import pytest

BK = 64; LA_FIN_ROWS = 8
TILE, P1, P2, FIN, END, SKIP = 0, 1, 2, 3, -1, 5

def sym_prefix(ty, tiles_x, epw):
    if epw == 1: f = ty * (ty - 1) // 2
    else:
        a = ty // 2
        f = a * (a - 1) if ty % 2 == 0 else a * a
    return ty * tiles_x - f

class Cfg:
    def __init__(s, n, epw, sym, grid_cap=152):
        s.n, s.epw, s.sym = n, epw, sym
        s.q = (n + BK - 1) // BK
        s.tiles_x = (n + 128 * epw - 1) // (128 * epw)
        s.tiles_y = (n + 127) // 128
        if sym:
            s.tiles_total = sum(s.tiles_x - min(s.tiles_x, y // epw) for y in range(s.tiles_y))
        else:
            s.tiles_total = s.tiles_x * s.tiles_y
        s.grid = min(grid_cap, s.tiles_total)
        s.has_rowP = (epw == 2 and sym)
        s.red = (epw == 1)   # int32 path (fp32 is !RED too; model epw==1 RED)
        s.ROW_BNW = 8192 // BK; s.COL_BM = 8192 * epw // BK
        s.base1 = s.round(0)['total']
        s.block = max(s.round(j)['total'] for j in range(1, s.q + 1))

    def round(s, j):
        n, q, E = s.n, s.q, s.epw
        r = {}
        r['p0'] = j * BK; r['p1'] = min(r['p0'] + BK, n)
        if j >= q:
            r.update(len_t=s.tiles_total, total=s.tiles_total, R=-1, C=-1, row_x0=0, col_y1=0, n_prio=0,
                     b1=s.tiles_total, b2=s.tiles_total, b3=s.tiles_total, n_p2row=0, n_p2col=0, n_fin=0)
            return r
        r['R'] = r['p0'] // 128; r['C'] = r['p0'] // (128 * E)
        r['row_x0'] = r['C'] if s.sym else 0
        r['col_y1'] = min(r['C'] * E + E, s.tiles_y) if s.sym else s.tiles_y
        r['n_prio'] = 0 if j == 0 else (s.tiles_x - r['row_x0']) + (r['col_y1'] - (1 if r['R'] < r['col_y1'] else 0))
        nrow = (n + s.ROW_BNW * E - 1) // (s.ROW_BNW * E); ncol = (n + s.COL_BM - 1) // s.COL_BM
        if s.sym:
            r['p2_row_first'] = r['p1'] // (s.ROW_BNW * E)
            r['n_p2row'] = max(0, nrow - r['p2_row_first'])
            r['n_p2col'] = (r['p0'] + s.COL_BM - 1) // s.COL_BM
        else:
            r['n_p2row'], r['n_p2col'] = nrow, ncol
        bs = (r['p0'] // (128 * E)) * (128 * E)
        w = r['p1'] - r['p0']
        r['n_fin'] = 0
        if s.sym and r['p0'] > 0:
            r['n_fin'] = (w + LA_FIN_ROWS - 1) // LA_FIN_ROWS if s.has_rowP else (1 if r['p0'] > bs else 0)
        if j == 0:
            r.update(len_t=0, b1=0, b2=0, b3=0, total=1 + r['n_p2row'] + r['n_p2col'] + r['n_fin'])
            return r
        r['len_t'] = r['n_prio'] + s.tiles_total
        G = s.grid
        r['b1'] = min(r['n_prio'] + 2 * G, r['len_t'])
        r['b2'] = min(r['b1'] + 4 * G, r['len_t'])
        r['b3'] = min(r['b2'] + 3 * G, r['len_t'])
        r['total'] = r['len_t'] + 1 + r['n_p2row'] + r['n_p2col'] + r['n_fin']
        return r

    def is_prio(s, r, y, x):
        return r['n_prio'] > 0 and ((y == r['R'] and x >= r['row_x0']) or (x == r['C'] and y < r['col_y1']))

    def stream_tile(s, r, j):
        if j < r['n_prio']:
            nr = s.tiles_x - r['row_x0']
            if j < nr: return (r['R'], r['row_x0'] + j)
            y = j - nr
            if y >= r['R']: y += 1
            return (y, r['C'])
        idx = j - r['n_prio']
        if not s.sym:
            y, x = idx // s.tiles_x, idx % s.tiles_x
        else:
            lo, hi = 0, s.tiles_y - 1
            while lo < hi:
                mid = (lo + hi + 1) >> 1
                if sym_prefix(mid, s.tiles_x, s.epw) <= idx: lo = mid
                else: hi = mid - 1
            y = lo; x = lo // s.epw + (idx - sym_prefix(lo, s.tiles_x, s.epw))
        return None if s.is_prio(r, y, x) else (y, x)

    def decode(s, item):
        if item < s.base1:
            r0 = s.round(0)
            if item == 0: return (P1, 0, 0)
            if item < 1 + r0['n_p2row'] + r0['n_p2col']: return (P2, 0, item - 1)
            return (SKIP, 0, 0)
        rel = item - s.base1
        j = 1 + rel // s.block; pos = rel % s.block
        if j > s.q: return (END, s.q, 0)
        r = s.round(j)
        if pos >= r['total']: return (SKIP, j, 0)
        n_p2 = r['n_p2row'] + r['n_p2col']
        if j < s.q:
            o1, o2, o3 = r['b1'], r['b2'] + 1, r['b3'] + 1 + n_p2
            if pos < o1: t = pos
            elif pos == o1: return (P1, j, 0)
            elif pos < o2: t = pos - 1
            elif pos < o2 + n_p2: return (P2, j, pos - o2)
            elif pos < o3: t = pos - 1 - n_p2
            elif pos < o3 + r['n_fin']: return (FIN, j, pos - o3)
            else: t = pos - 1 - n_p2 - r['n_fin']
            tl = s.stream_tile(r, t)
            return (SKIP, j, 0) if tl is None else (TILE, j - 1, tl)
        tl = s.stream_tile(r, pos)
        return (TILE, j - 1, tl)

def simulate(cfg, seed, task_in_c, blocking=False):
    rng = random.Random(seed)
    G = cfg.grid; q = cfg.q
    items = [0]
    cnt = {}  # (r, f) -> value
    def C(r, f): return cnt.get((r, f), 0)
    def inc(r, f): cnt[(r, f)] = C(r, f) + 1
    tile_round = {}
    tiles_done_round = {}   # (round, tile) processed count for coverage check
    tasks_done = set()
    class CTA: pass
    ctas = []
    for c in range(G):
        t = CTA()
        t.claimed = []; t.issued = 0; t.hold = -1; t.stop = False; t.ok = True
        t.queue = []  # reserved items
        t.c_next = 0; t.cs_free = True; t.c_issued = []  # C loads issued for tile ordinals (slot indices)
        t.ready = -1
        t.empty = set(); t.cdone = set(); t.full = set()
        t.cfree = 0   # number of cfree arrivals
        t.full_c = 0  # C loads landed
        t.pi = 0; t.pstate = 'prologue'
        t.ci = 0; t.cstate = 'wait_full'; t.ct = 0; t.cdone_flag = False
        t.done_p = False; t.done_c = False
        ctas.append(t)
    def next_item(t):
        if t.queue: return t.queue.pop(0)
        v = items[0]; items[0] += 1; return v
    def panels_ready(t, k):
        if k <= t.ready: return True
        r = cfg.round(k)
        if C(k, 3) < 1 + r['n_p2row'] + r['n_p2col'] + r['n_fin']: return False
        t.ready = k; return True
    def issue_slots(t):
        while t.issued < len(t.claimed):
            kind, rnd, info = t.claimed[t.issued]
            if kind == TILE and not panels_ready(t, rnd): return
            t.full.add(t.issued); t.issued += 1
    def issue_c(t):
        if cfg.red: return
        while t.c_next < len(t.claimed) and t.claimed[t.c_next][0] != TILE: t.c_next += 1
        if not t.cs_free or t.c_next >= len(t.claimed): return
        kind, k, tl = t.claimed[t.c_next]
        if tile_round.get(tl, 0) < k: return
        t.c_issued.append(t.c_next); t.cs_free = False; t.c_next += 1
        t.full_c += 1
    def progress(t):
        before = (t.issued, len(t.c_issued))
        issue_slots(t); issue_c(t)
        return (t.issued, len(t.c_issued)) != before
    def claim(t):
        while True:
            kind, rnd, info = cfg.decode(next_item(t))
            if kind != SKIP: break
        t.claimed.append((kind, rnd, info))
        if kind == END: t.stop = True
        elif kind != TILE and not task_in_c: t.hold = len(t.claimed) - 1
        progress(t)
    def prod_step(t):
        if t.done_p: return False
        if blocking and t.pstate != 'prologue' and t.issued < len(t.claimed):
            return progress(t)  # the earlier design: stuck in claim() until the pending slot can be issued
        if t.pstate == 'prologue':
            v = items[0]; items[0] += 2; t.queue = [v, v + 1]
            claim(t)
            if not t.stop and t.hold < 0: claim(t)
            t.pstate = 'top'; return True
        i = t.pi
        if t.pstate == 'top':
            kind = t.claimed[i][0]
            if kind == END:
                moved = progress(t)
                if t.issued == len(t.claimed): t.done_p = True; return True
                return moved
            t.pstate = 'wait_empty'; return True
        if t.pstate == 'wait_empty':
            if i in t.empty:
                if not t.stop and t.hold < 0 and len(t.claimed) < i + 3: claim(t)
                t.pstate = 'wait_cdone'; return True
            return progress(t)
        if t.pstate == 'wait_cdone':
            if i in t.cdone:
                kind, k, info = t.claimed[i]
                if kind == TILE:
                    if cfg.red: t.cfree += 1
                    else: t.cs_free = True
                    # publish
                    assert tile_round.get(info, 0) == k or cfg.red, ("tile round order", info, k, tile_round.get(info, 0))
                    if not cfg.red: tile_round[info] = k + 1
                    tiles_done_round[(k, info)] = tiles_done_round.get((k, info), 0) + 1
                    inc(k, 4)
                    if k + 1 < q:
                        r = cfg.round(k + 1)
                        if cfg.is_prio(r, info[0], info[1]): inc(k + 1, 0)
                    progress(t)
                elif not task_in_c:
                    t.hold = -1
                    while not t.stop and t.hold < 0 and len(t.claimed) < i + 3: claim(t)
                t.pi += 1; t.pstate = 'top'; return True
            return progress(t)
    def cons_step(t):
        if t.done_c: return False
        j = t.ci
        if t.cstate == 'wait_full':
            if j not in t.full: return False
            kind, rnd, info = t.claimed[j]
            if kind == END: t.done_c = True; return True
            t.cur = (kind, rnd, info)
            if kind == TILE:
                # panels of round rnd must be complete (TMA read happened at issue)
                r = cfg.round(rnd)
                assert C(rnd, 3) >= 1 + r['n_p2row'] + r['n_p2col'] + r['n_fin'], "tile before its panels"
                t.empty.add(j)
                t.cstate = 'tile_epi'
            else:
                if task_in_c: t.empty.add(j)
                t.cstate = 'task_cfree' if task_in_c else 'task_dep'
            return True
        kind, rnd, info = t.cur
        if t.cstate == 'tile_epi':
            if cfg.red:
                if t.ct > 0 and t.cfree < t.ct: return False
            else:
                if t.full_c <= t.ct: return False
                # the C load of this tile happened only once its previous round was written
                assert t.c_issued[t.ct] == j
            t.ct += 1; t.cdone.add(j); t.ci += 1; t.cstate = 'wait_full'; return True
        if t.cstate == 'task_cfree':
            if t.ct > 0 and t.cfree < t.ct: return False
            t.cstate = 'task_dep'; return True
        if t.cstate == 'task_dep':
            r = cfg.round(rnd)
            if kind == P1:
                if rnd >= 1 and C(rnd, 0) < r['n_prio']: return False
                if rnd >= 2 and C(rnd - 2, 4) < cfg.tiles_total: return False
            elif kind == P2:
                if C(rnd, 1) < 1: return False
            else:
                if C(rnd, 2) < r['n_p2row'] + r['n_p2col']: return False
            # run the task
            if kind == P1: inc(rnd, 1)
            elif kind == P2: inc(rnd, 2)
            inc(rnd, 3)
            tasks_done.add((kind, rnd, info))
            if not task_in_c: t.empty.add(j)
            t.cdone.add(j); t.ci += 1; t.cstate = 'wait_full'; return True
    steps = 0; idle = 0
    while True:
        live = [t for t in ctas if not (t.done_p and t.done_c)]
        if not live: break
        moved = False
        order = list(range(len(live) * 2)); rng.shuffle(order)
        for o in order:
            t = live[o // 2]
            if (prod_step(t) if o % 2 == 0 else cons_step(t)):
                moved = True; break
        steps += 1
        if not moved:
            raise RuntimeError(f"deadlock after {steps} steps: " + "; ".join(
                f"cta{ctas.index(t)} p={t.pstate}@{t.pi} issued={t.issued}/{len(t.claimed)} c={t.cstate}@{t.ci}"
                for t in live))
    # coverage: every tile of every round exactly once, every task once
    for k in range(q if q > 1 else 0):
        pass
    exp_tiles = set()
    for y in range(cfg.tiles_y):
        for x in range(cfg.tiles_x):
            if not cfg.sym or x >= y // cfg.epw: exp_tiles.add((y, x))
    for k in range(q):
        for tl in exp_tiles:
            assert tiles_done_round.get((k, tl), 0) == 1, ("tile coverage", k, tl, tiles_done_round.get((k, tl), 0))
    for j in range(q):
        r = cfg.round(j)
        assert (P1, j, 0) in tasks_done
        for i in range(r['n_p2row'] + r['n_p2col']): assert (P2, j, i) in tasks_done
        for i in range(r['n_fin']): assert (FIN, j, i) in tasks_done, ("fin", j, i)
    return steps



CASES = [(n, epw, sym, cap) for n in (65, 129, 300, 777, 1000) for epw in (1, 2) for sym in (0, 1)
         for cap in (2, 3, 7, 152)]


@pytest.mark.parametrize("n,epw,sym,cap", CASES)
def test_schedule_completes_in_order_and_covers_everything(n, epw, sym, cap):
    cfg = Cfg(n, epw, sym, cap)
    if cfg.q < 2:
        pytest.skip("one round: no Phase 3")
    for seed in range(2):
        simulate(cfg, seed * 7919 + n + cap, epw == 1)


def test_a_blocking_producer_can_stall():
    stalls = 0
    for n in (65, 129, 300):
        for epw in (1, 2):
            for cap in (2, 3):
                for seed in range(3):
                    try:
                        simulate(Cfg(n, epw, 0, cap), seed, epw == 1, blocking=True)
                    except RuntimeError:
                        stalls += 1
    assert stalls > 0
