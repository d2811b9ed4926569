"""Team-cooperative form of a class program (the tier for large classes).

A team of T lanes (one to sixteen warps) evaluates ONE primitive quartet at a
time: the Phase-1 graph is cut into waves of mutually independent nodes,
taken in DSA order (FusionRCG Eq. 7) by a bounded-width list scheduler; a
wave is one or more steps of ilp nodes per lane (several steps only for
teams of 256 or more lanes), and a team barrier separates waves.  Phase 2
is scheduled the same way, with its operations in their liveness-friendly
build order as priority.  Values live in one slot space
per team (not per lane), so a class whose sequential PeakLive (Eq. 4) is
thousands of values still fits in shared memory; the accumulator bank H is
addressed separately (shared memory when it fits, else a team-private global
region).

Phase-1 descriptor (uint16 x8): dst slot (0xFFFF: not kept), h = target + 1
(0: none), operand slots s0..s4, and meta:
  bits 0-3   6 side + axis  (coefficient rows of P-A / W-P or Q-C / W-Q)
  bits 4-8   k (second Obara-Saika term; for a base node the Boys order m)
  bits 9-12  k3 (cross term)
  bit 13     side (0 bra, 1 ket)
  bit 14     base node [00|00]^(m)
  bit 15     no-op
Phase-2 operand ids: id < nh is accumulator H[id]; id >= nh is value slot
id - nh.
Phase-2 descriptor kinds: 0 HRR, 1 LIN (n <= 4), 2 STORE, 3 no-op; a
transform row of more than four terms becomes a chain of LIN descriptors in
successive waves, each continuing with 1.0 x the previous partial sum.
"""
from __future__ import annotations

from dataclasses import dataclass
import heapq

import numpy as np

from .encode import coef_table

NOP1 = np.array([0xFFFF, 0, 0, 0x8000 << 16], dtype=np.uint32)
NOP2 = np.array([3, 0, 0, 0], dtype=np.uint32)
MAX_ID = 65535


def wave_schedule(parents, priority, width):
    """Bounded-width list scheduling: each wave takes up to ``width`` ready
    nodes with the smallest priority.  parents[v] = list of node ids."""
    n = len(parents)
    cons = [[] for _ in range(n)]
    npar = [0] * n
    for v, ps in enumerate(parents):
        ps = set(ps)
        npar[v] = len(ps)
        for p in ps:
            cons[p].append(v)
    ready = [(priority[v], v) for v in range(n) if npar[v] == 0]
    heapq.heapify(ready)
    waves = []
    while ready:
        cur = []
        while ready and len(cur) < width:
            cur.append(heapq.heappop(ready)[1])
        for v in cur:
            for c in cons[v]:
                npar[c] -= 1
                if npar[c] == 0:
                    heapq.heappush(ready, (priority[c], c))
        waves.append(cur)
    assert sum(len(w) for w in waves) == n, "cycle in graph"
    return waves


def allocate_over_waves(parents, waves, needs_slot, first_slot=0, pinned_until_end=()):
    """Slots for wave-synchronous execution: a value written in wave b and
    last read in wave d keeps its slot through wave d; a slot is reused only
    by a value born in a later wave.  Lowest free slot first."""
    n = len(parents)
    wave_of = np.zeros(n, dtype=np.int64)
    for w, vs in enumerate(waves):
        for v in vs:
            wave_of[v] = w
    last = wave_of.copy()
    for v, ps in enumerate(parents):
        for p in ps:
            last[p] = max(last[p], wave_of[v])
    for v in pinned_until_end:
        last[v] = len(waves)
    slot = np.full(n, -1, dtype=np.int64)
    free = []
    nxt = first_slot
    release_at = [[] for _ in range(len(waves) + 2)]
    for w, vs in enumerate(waves):
        for s in release_at[w]:
            heapq.heappush(free, s)
        for v in vs:
            if not needs_slot[v]:
                continue
            if free:
                slot[v] = heapq.heappop(free)
            else:
                slot[v] = nxt
                nxt += 1
            release_at[last[v] + 1].append(int(slot[v]))
    return slot, nxt - first_slot


ILP = 2  # default nodes per lane per step (independent chains per lane)


@dataclass
class CoopProgram:
    T: int
    ilp: int
    ph1: np.ndarray        # uint32 [sum steps * T, 4]
    steps1: np.ndarray     # uint32 [nwave1] steps of each wave
    ph2: np.ndarray
    steps2: np.ndarray
    nh: int
    nslot: int             # value slots (ids nh .. nh + nslot - 1)
    L: int
    out_dims: tuple
    eff1: float            # busy lanes / lane slots, Phase 1
    eff2: float


PREFETCH_STEPS = 2  # no-op steps after the last wave: the executor loads ahead


def _pack(waves, rows_of, T, nop, ilp, shape_of=None):
    """A step is ilp * T descriptors: lane l takes descriptors ilp*l .. ilp*l +
    ilp - 1 of the step, so a wave of n nodes spreads over the lanes first.
    shape_of(descriptor): the nodes of a wave are independent, so they are
    placed in order of their shape (which optional terms they evaluate):
    the 32 lanes of a warp then mostly share one shape, and a warp issues the
    optional FP64 instructions only when some lane needs them."""
    ILP = ilp
    W = ILP * T
    steps = []
    out = []
    for vs in waves:
        st = (len(vs) + W - 1) // W
        steps.append(st)
        block = np.tile(nop, (st * W, 1))
        rows = [rows_of(v) for v in vs]
        if shape_of is not None:
            rows.sort(key=shape_of)   # stable: DSA order within a shape
        for k, row in enumerate(rows):
            s, r = divmod(k, W)
            lane, j = r % T, r // T       # fill every lane's first node before second nodes
            block[s * W + lane * ILP + j] = row
        out.append(block)
    out.append(np.tile(nop, (PREFETCH_STEPS * W, 1)))
    arr = np.concatenate(out)
    return arr.astype(np.uint32), np.array(steps, dtype=np.uint32)


def build(prog, T=128, ilp=ILP, wave_steps=1):
    """CoopProgram of a class program for teams of T lanes taking ilp nodes
    per step; a wave (the nodes between two team barriers) holds up to
    wave_steps steps of mutually independent nodes."""
    g = prog.g
    nh = prog.nh
    # ---------------- Phase 1
    order_pos = np.empty(len(g), dtype=np.int64)
    order_pos[np.array(prog.order, dtype=np.int64)] = np.arange(len(g))
    par1 = [[p for _, p in ts] for ts in g.terms]
    waves1 = wave_schedule(par1, order_pos, ilp * T * wave_steps)
    consumed = np.zeros(len(g), dtype=bool)
    for ps in par1:
        for p in ps:
            consumed[p] = True
    slot1, nslot1 = allocate_over_waves(par1, waves1, consumed)

    def row1(v):
        ts = g.terms[v]
        dst = int(slot1[v]) if consumed[v] else 0xFFFF
        h = g.target.get(v)
        src = [0] * 5
        meta = 0
        if not ts:
            meta = (1 << 14) | (g.keys[v][2] << 4)
        for (kind, val), p in ts:
            s_ = int(slot1[p])
            if kind in ("PA", "QC"):
                side = 0 if kind == "PA" else 1
                src[0] = s_
                meta |= (6 * side + val) | (side << 13)
            elif kind in ("WP", "WQ"):
                src[1] = s_
            elif kind in ("c1z", "c1e"):
                src[2] = s_
                meta |= val << 4
            elif kind in ("c2z", "c2e"):
                src[3] = s_
            elif kind == "c3":
                src[4] = s_
                meta |= val << 9
        return np.array([dst | ((h + 1) << 16 if h is not None else 0), src[0] | (src[1] << 16),
                         src[2] | (src[3] << 16), src[4] | (meta << 16)], dtype=np.uint32)

    def shape1(row):
        # base node; c1/c2 pair present; c3 term present
        meta = int(row[3]) >> 16
        return ((meta >> 14) & 1, ((meta >> 4) & 31) > 0, ((meta >> 9) & 15) > 0)

    ph1, steps1 = _pack(waves1, row1, T, NOP1, ilp, shape1)

    # ---------------- Phase 2: graph of operations and output stores
    p2 = prog.p2
    ctab = {c: i for i, c in enumerate(coef_table())}
    # node ids: 0..nh-1 = H inputs; then one node per operation chunk; then stores
    nodes = []      # (kind, payload)
    parents = []
    val_node = {i: i for i in range(nh)}   # value id -> node producing it
    for i in range(nh):
        nodes.append(("h", i))
        parents.append([])
    for op in p2.ops:
        if op[0] == "hrr":
            _, d, hi, sym_i, lo = op
            nid = len(nodes)
            nodes.append(("hrr", (hi, lo, sym_i)))
            parents.append([val_node[hi], val_node[lo]])
            val_node[d] = nid
        else:
            # rows of more than four terms: the first descriptor sums four,
            # each further one adds 1.0 x the running sum and up to three more
            _, d, terms = op
            prev = None
            rest = list(terms)
            while rest:
                take = 4 if prev is None else 3
                chunk, rest = rest[:take], rest[take:]
                nid = len(nodes)
                nodes.append(("lin", (chunk, prev)))
                ps = [val_node[s] for _, s in chunk]
                if prev is not None:
                    ps.append(prev)
                parents.append(ps)
                prev = nid
            val_node[d] = prev
    store_nodes = []
    for k, v in enumerate(p2.outputs):
        nid = len(nodes)
        nodes.append(("store", (k, v)))
        parents.append([val_node[v]])
        store_nodes.append(nid)
    n2 = len(nodes)
    prio = np.arange(n2, dtype=np.int64)
    # stores go right after their value: priority of the producer
    for nid in store_nodes:
        prio[nid] = parents[nid][0]
    # H inputs are not scheduled (they are read in place)
    work = [v for v in range(n2) if nodes[v][0] != "h"]
    pos = {v: i for i, v in enumerate(work)}
    par_list = [[pos[p] for p in parents[v] if nodes[p][0] != "h"] for v in work]
    waves2 = wave_schedule(par_list, np.array([prio[v] for v in work]), ilp * T * wave_steps)
    waves2 = [[work[i] for i in w] for w in waves2]
    needs = np.zeros(n2, dtype=bool)
    for v in range(n2):
        if nodes[v][0] in ("hrr", "lin"):
            needs[v] = True
    # slot allocation over the waves (H inputs keep their own ids)
    sched = [v for w in waves2 for v in w]
    loc = {v: i for i, v in enumerate(sched)}
    p_loc = [[loc[p] for p in parents[v] if p in loc] for v in sched]
    w_loc = []
    c = 0
    for w in waves2:
        w_loc.append(list(range(c, c + len(w))))
        c += len(w)
    slot_l, nslot2 = allocate_over_waves(p_loc, w_loc, np.array([needs[v] for v in sched]))
    slot2 = {v: int(slot_l[loc[v]]) for v in sched}

    def oid(node):
        # operand id of a node's value: H index or nh + slot
        return node if nodes[node][0] == "h" else nh + slot2[node]

    def row2(v):
        kind, pl = nodes[v]
        if kind == "hrr":
            hi, lo, (sym, i) = pl
            return np.array([0 | (oid(v) << 16), oid(val_node[hi]) | (oid(val_node[lo]) << 16),
                             i + (3 if sym == "CD" else 0), 0], dtype=np.uint32)
        if kind == "lin":
            chunk, prev = pl
            terms = [(float(cf), oid(val_node[s])) for cf, s in chunk]
            if prev is not None:
                terms.append((1.0, oid(prev)))
            n = len(terms)
            ss = [x for _, x in terms] + [0] * (4 - n)
            cc = [ctab[cf] for cf, _ in terms] + [0] * (4 - n)
            return np.array([1 | (n << 2) | (oid(v) << 16), ss[0] | (ss[1] << 16), ss[2] | (ss[3] << 16),
                             cc[0] | (cc[1] << 8) | (cc[2] << 16) | (cc[3] << 24)], dtype=np.uint32)
        k, val = pl
        i = np.unravel_index(k, p2.out_dims)
        return np.array([2 | (oid(val_node[val]) << 16), k,
                         int(i[0]) | (int(i[1]) << 8) | (int(i[2]) << 16) | (int(i[3]) << 24), 0], dtype=np.uint32)

    def shape2(row):
        # kind (HRR, linear combination, store) and number of terms
        return (int(row[0]) & 3, (int(row[0]) >> 2) & 7)

    ph2, steps2 = _pack(waves2, row2, T, NOP2, ilp, shape2)
    nslot = max(int(nslot1), int(nslot2))
    if nslot >= 0xFFFF or nh + nslot > MAX_ID:
        raise ValueError("class {} needs {} ids".format(prog.ls, nh + nslot))
    eff1 = len(g) / max(1, int(steps1.sum()) * T * ilp)
    eff2 = len(sched) / max(1, int(steps2.sum()) * T * ilp)
    assert ph1.shape[0] == (int(steps1.sum()) + PREFETCH_STEPS) * T * ilp
    return CoopProgram(T, ilp, ph1, steps1, ph2, steps2, nh, nslot, prog.L, tuple(p2.out_dims), eff1, eff2)


ROW_BYTES = 56 * 8           # one primitive quartet's coefficient row (executor constant)
DEEP_ROWS = 32               # rows per team for deep contractions (one per lane of a warp)
SHALLOW_ROWS = 12            # rows per team for contractions of at most 12 primitive quartets
SMEM_PER_SM = 228 * 1024
SHAPES = ((32, 2), (64, 2), (128, 2), (128, 4))


def _score(cp, rows):
    """Useful FP64 work per SM of a built shape: resident warps (shared
    memory for the team's rows, value slots and, when it fits, H; at most
    16 warps), times the lane efficiency of the waves, times a
    latency-hiding factor for the independent chains per SM sub-partition
    (warps / 4 x nodes per lane, saturating at 4: measured, two warps of two
    nodes each per sub-partition already cover the FP64 latency, and four
    nodes per lane then only cost lane efficiency).  None if it does not
    fit."""
    vals = cp.nslot * 8 + rows * ROW_BYTES
    with_h = vals + cp.nh * 8
    per_team = with_h if with_h <= 227 * 1024 else vals
    if per_team > 227 * 1024:
        return None
    # registers: 4 nodes per lane need ~230 registers (256 threads per SM)
    max_threads = 256 if cp.ilp == 4 else 512
    teams = max(1, min(SMEM_PER_SM // (per_team + 1024), max_threads // cp.T))
    warps = min(teams * cp.T // 32, max_threads // 32)
    eff = 0.5 * (cp.eff1 + cp.eff2) * 0.2 + cp.eff1 * 0.8
    chains = warps / 4.0 * cp.ilp
    return warps * eff * min(1.0, chains / 4.0)


WIDE_SHAPES = ((256, 2), (256, 4))
# sixteen warps on one live set: 512 lanes, two nodes per lane (the register
# file holds 128 registers for each of 512 threads)
WIDEST_SHAPE = (512, 2)
WAVE_NODES_MAX = 2048   # nodes in a multi-step wave of a 512-lane team


def _teams_per_sm(cp, rows, h_in_smem=True):
    vals = cp.nslot * 8 + rows * ROW_BYTES
    with_h = vals + cp.nh * 8
    per_team = with_h if h_in_smem and with_h <= 227 * 1024 else vals
    return SMEM_PER_SM // (per_team + 1024)


def _wide_waves(prog, cp, rows):
    """A team of 256 or more lanes is alone on its SM and meets a barrier
    after every step; waves of up to four steps of independent nodes cut the
    barriers about fourfold (measured: (gg|gg) 0.45 -> 0.52 of the FP64 rate
    with 256 lanes) at the cost of a larger live set.  Take the widest of 4
    and 2 steps that keeps the teams per SM, with at most WAVE_NODES_MAX nodes
    in a wave (512 lanes x 2 nodes x 2 steps: the live set and the barrier
    count of the 256-lane, 4-step waves); narrower teams keep one step per
    wave (measured: the larger live set costs them residency or lane
    efficiency)."""
    if cp is None or cp.T < 256:
        return cp
    for k in (4, 2):
        if cp.T == 512 and cp.T * cp.ilp * k > WAVE_NODES_MAX:
            continue
        ck = build(prog, cp.T, cp.ilp, k)
        if _score(ck, rows) is not None and _teams_per_sm(ck, rows) >= _teams_per_sm(cp, rows):
            return ck
    return cp


def choose_both(prog, shapes=SHAPES):
    """(deep, shallow): the best (team size, nodes per lane) shape when a
    team holds DEEP_ROWS coefficient rows, and when it holds SHALLOW_ROWS
    (shallow contractions: fewer rows leave shared memory for more teams).
    Classes whose 128-lane team is alone on an SM also try one 256-lane team
    (eight warps on the same shared-memory live set), and those whose
    256-lane team is alone even with H in global memory one 512-lane team
    (sixteen warps)."""
    built = [build(prog, T, ilp) for T, ilp in shapes]
    if any(cp.T == 128 and _teams_per_sm(cp, DEEP_ROWS) <= 1 for cp in built):
        built += [build(prog, T, ilp) for T, ilp in WIDE_SHAPES]
        # a 512-lane team only where a 256-lane team is alone on its SM even
        # with H in global memory (the runtime then holds eight warps per SM,
        # the 512-lane team sixteen).  Measured with K per shell from
        # {1, 3, 6}: (gg|gg) 0.546 -> 0.602 of the FP64 rate, (gg|gf) 0.521
        # -> 0.575; where two 256-lane teams (or three 128-lane ones) fit, the
        # wider team only costs lane efficiency ((fg|dg) 0.638 -> 0.466).
        if any(cp.T == 256 and cp.ilp == 2 and _teams_per_sm(cp, DEEP_ROWS, h_in_smem=False) <= 1
               for cp in built):
            built.append(build(prog, *WIDEST_SHAPE))
    out = []
    for rows in (DEEP_ROWS, SHALLOW_ROWS):
        scored = [(sc, k) for k, cp in enumerate(built) for sc in [_score(cp, rows)] if sc is not None]
        out.append(_wide_waves(prog, built[max(scored)[1]], rows) if scored else None)
    return tuple(out)


def choose(prog, shapes=SHAPES):
    """The best shape for deep contractions (see choose_both)."""
    return choose_both(prog, shapes)[0]
