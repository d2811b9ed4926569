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


def _consumer_lists(parents, n):
    """Distinct-parent counts and consumer lists of a node list."""
    cons = [[] for _ in range(n)]
    npar = [0] * n
    for v, ps in enumerate(parents):
        ps = set(ps)
        npar[v] = len(ps)
        for p in ps:
            cons[p].append(v)
    return cons, npar


def _waves(cons, npar, priority, width, lag=1):
    """Bounded-width list scheduling over consumer lists (npar is consumed):
    each wave takes up to ``width`` ready nodes, smallest (priority, node)
    first, in that order.  A node whose last parent is placed in wave w
    becomes ready in wave w + lag: lag 1 for waves separated by a full team
    barrier, lag 2 for split barriers (a lane may start wave w + 1 while
    others still run wave w, so wave w + 1 reads nothing wave w writes)."""
    ready = [(priority[v], v) for v in range(len(npar)) if npar[v] == 0]
    heapq.heapify(ready)
    pop, push = heapq.heappop, heapq.heappush
    pending = [[] for _ in range(lag)]   # pending[j]: ready j + 1 waves from now
    waves = []
    placed, n = 0, len(npar)
    while placed < n:
        for v in pending.pop(0):
            push(ready, (priority[v], v))
        pending.append([])
        if not ready:
            assert any(pending), "cycle in graph"
            waves.append([])
            continue
        cur = [pop(ready)[1] for _ in range(min(width, len(ready)))]
        for v in cur:
            for c in cons[v]:
                npar[c] -= 1
                if npar[c] == 0:
                    pending[lag - 1].append(c)
        waves.append(cur)
        placed += len(cur)
    return waves


def wave_schedule(parents, priority, width, lag=1):
    """Bounded-width list scheduling: each wave takes up to ``width`` ready
    nodes with the smallest priority; a node's parents lie at least ``lag``
    waves before it.  parents[v] = list of node ids."""
    n = len(parents)
    cons, npar = _consumer_lists(parents, n)
    return _waves(cons, npar, [int(x) for x in priority], width, lag)


def _allocate(wave_of, last, needs_slot, order, first_slot=0, lag=1):
    """Slot allocation over waves for nodes taken in ``order`` (wave by wave):
    a value written in wave b and last read in wave d keeps its slot through
    wave d + lag - 1; a slot is reused only by a value born in wave d + lag
    or later (lag 2: a lane may still be reading it in wave d while another
    writes wave d + 1).  Lowest free slot first."""
    n = len(wave_of)
    slot = np.full(n, -1, dtype=np.int64)
    free = []
    nxt = first_slot
    nw = int(wave_of.max()) + 1 if n else 0
    release_at = [[] for _ in range(max(nw, int(last.max()) + 1 if n else 0) + 1 + lag)]
    pop, push = heapq.heappop, heapq.heappush
    cur_w = -1
    wl = wave_of.tolist()
    ll = last.tolist()
    nl = needs_slot.tolist()
    out = [-1] * n
    for v in order:
        w = wl[v]
        while cur_w < w:
            cur_w += 1
            for s in release_at[cur_w]:
                push(free, s)
        if not nl[v]:
            continue
        if free:
            s = pop(free)
        else:
            s = nxt
            nxt += 1
        out[v] = s
        release_at[ll[v] + lag].append(s)
    slot[:] = out
    return slot, nxt - first_slot


NBANK = 16  # 8-byte shared-memory words: 32 four-byte banks serve 16 words per half-warp


def _allocate_banked(wave_of, last, needs_slot, order, groups, fixed=None, lag=1):
    """Slot allocation as _allocate, but a value takes, among the free slots,
    one whose shared-memory bank its accesses share with the fewest values
    already placed.  A 64-bit shared access of a warp is served in two
    half-warp passes, each needing as many wavefronts as the most values it
    finds in one bank (8-byte word index mod 16); ``groups[v]`` lists the
    access groups (one per half-warp instruction) value v belongs to.  The
    choice never creates a slot while one is free, so the slot count equals
    _allocate's.  ``fixed``: (group, bank) pairs of operands outside the
    slots (accumulators in shared memory) already in a group."""
    n = len(wave_of)
    ng = 1 + max((max(g) for g in groups if len(g)), default=-1)
    if fixed is not None and len(fixed):
        ng = max(ng, 1 + int(fixed[:, 0].max()))
    hist = np.zeros((max(1, ng), NBANK), dtype=np.int32)
    if fixed is not None and len(fixed):
        np.add.at(hist, (fixed[:, 0], fixed[:, 1]), 1)
    free = [[] for _ in range(NBANK)]
    nxt = 0
    nw = int(wave_of.max()) + 1 if n else 0
    release_at = [[] for _ in range(max(nw, int(last.max()) + 1 if n else 0) + 1 + lag)]
    pop, push = heapq.heappop, heapq.heappush
    cur_w = -1
    wl = wave_of.tolist()
    ll = last.tolist()
    nl = needs_slot.tolist()
    out = [-1] * n
    big = np.int64(1) << 40
    for v in order:
        w = wl[v]
        while cur_w < w:
            cur_w += 1
            for s in release_at[cur_w]:
                push(free[s % NBANK], s)
        if not nl[v]:
            continue
        g = groups[v]
        tops = np.array([f[0] if f else big for f in free], dtype=np.int64)
        if len(g):
            h = hist[g]
            # groups whose most loaded bank this choice would deepen
            cost = (h >= h.max(1)[:, None]).sum(0).astype(np.int64)
        else:
            cost = np.zeros(NBANK, dtype=np.int64)
        # fewest conflicts first, then the lowest slot
        key = np.where(tops == big, big, cost * (np.int64(1) << 32) + tops)
        b = int(np.argmin(key))
        if key[b] == big:
            s = nxt
            nxt += 1
        else:
            s = pop(free[b])
        if len(g):
            hist[g, s % NBANK] += 1
        out[v] = s
        release_at[ll[v] + lag].append(s)
    return np.asarray(out, dtype=np.int64), nxt


def _lifetimes(parents, waves, pinned_until_end=()):
    """Wave of every node and the last wave that reads it (its own wave if
    nothing does; pinned nodes: past the last wave)."""
    n = len(parents)
    wave_of = np.zeros(n, dtype=np.int64)
    for w, vs in enumerate(waves):
        wave_of[np.asarray(vs, dtype=np.int64)] = w
    last = wave_of.copy()
    src = [p for ps in parents for p in ps]
    if src:
        dst = np.repeat(np.arange(n, dtype=np.int64), [len(ps) for ps in parents])
        np.maximum.at(last, np.asarray(src, dtype=np.int64), wave_of[dst])
    for v in pinned_until_end:
        last[v] = len(waves)
    return wave_of, last


def allocate_over_waves(parents, waves, needs_slot, first_slot=0, pinned_until_end=(), lag=1):
    """Slots for wave-synchronous execution: a value written in wave b and
    last read in wave d keeps its slot through wave d + lag - 1; a slot is
    reused only by a value born in wave d + lag or later.  Lowest free slot
    first."""
    wave_of, last = _lifetimes(parents, waves, pinned_until_end)
    order = [v for vs in waves for v in vs]
    return _allocate(wave_of, last, np.asarray(needs_slot, dtype=bool), order, first_slot, lag)


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
    lag: int = 1           # 1: a full team barrier after every wave; 2: split
                           # barriers (wave w waits for wave w - 2 only)


PREFETCH_STEPS = 2  # no-op steps after the last wave: the executor loads ahead


def _pack(waves, rows, T, nop, ilp, shape):
    """A step is ilp * T descriptors: lane l takes descriptors ilp*l .. ilp*l +
    ilp - 1 of the step, so a wave of n nodes spreads over the lanes first
    (every lane's first node before any second node).  rows[v] is node v's
    descriptor; shape[v] a small integer naming which optional terms it
    evaluates.  The nodes of a wave are independent, so they are placed in
    order of their shape (stable: DSA order within a shape): the 32 lanes of
    a warp then mostly share one shape, and a warp issues the optional FP64
    instructions only when some lane needs them."""
    W = ilp * T
    sizes = np.array([len(w) for w in waves], dtype=np.int64)
    steps = (sizes + W - 1) // W
    total = (int(steps.sum()) + PREFETCH_STEPS) * W
    arr = np.tile(nop, (total, 1))
    if len(waves):
        idx = np.concatenate([np.asarray(w, dtype=np.int64) for w in waves])
        wave_id = np.repeat(np.arange(len(waves)), sizes)
        idx = idx[np.lexsort((np.arange(idx.size), shape[idx], wave_id))]
        k = np.arange(idx.size) - np.repeat(np.cumsum(sizes) - sizes, sizes)
        s, r = np.divmod(k, W)
        base = np.repeat(np.cumsum(steps * W) - steps * W, sizes)
        arr[base + s * W + (r % T) * ilp + r // T] = rows[idx]
    return arr.astype(np.uint32), steps.astype(np.uint32)


class _Static:
    """The parts of a class program's cooperative form that do not depend on
    the team shape, built once per program: Phase-1 parents and descriptor
    templates, and the Phase-2 graph of operations and output stores with
    its descriptor templates."""

    def __init__(self, prog):
        g = prog.g
        nh = prog.nh
        n = len(g)
        self.nh = nh
        self.n1 = n
        # ---------------- Phase 1
        order_pos = np.empty(n, dtype=np.int64)
        order_pos[np.array(prog.order, dtype=np.int64)] = np.arange(n)
        self.prio1 = order_pos.tolist()
        par1 = [[p for _, p in ts] for ts in g.terms]
        self.par1 = par1
        self.cons1, self.npar1 = _consumer_lists(par1, n)
        consumed = np.zeros(n, dtype=bool)
        for ps in par1:
            for p in ps:
                consumed[p] = True
        self.consumed = consumed
        # descriptor template: word 0 high half (h + 1), the meta field, and
        # the node feeding each of the five operand positions (-1: none)
        hword = np.zeros(n, dtype=np.int64)
        meta = np.zeros(n, dtype=np.int64)
        src = np.full((n, 5), -1, dtype=np.int64)
        for v, ts in enumerate(g.terms):
            h = g.target.get(v)
            if h is not None:
                hword[v] = (h + 1) << 16
            m = 0
            if not ts:
                m = (1 << 14) | (g.keys[v][2] << 4)
            for (kind, val), p in ts:
                if kind in ("PA", "QC"):
                    side = 0 if kind == "PA" else 1
                    src[v, 0] = p
                    m |= (6 * side + val) | (side << 13)
                elif kind in ("WP", "WQ"):
                    src[v, 1] = p
                elif kind in ("c1z", "c1e"):
                    src[v, 2] = p
                    m |= val << 4
                elif kind in ("c2z", "c2e"):
                    src[v, 3] = p
                elif kind == "c3":
                    src[v, 4] = p
                    m |= val << 9
            meta[v] = m
        self.hword, self.meta1, self.src1 = hword, meta, src
        # shape of a Phase-1 node: base node; c1/c2 pair present; c3 present
        self.shape1 = (((meta >> 14) & 1) * 4 + (((meta >> 4) & 31) > 0) * 2
                       + (((meta >> 9) & 15) > 0)).astype(np.int64)
        # ---------------- Phase 2: graph of operations and output stores
        p2 = prog.p2
        ctab = {c: i for i, c in enumerate(coef_table())}
        # node ids: 0..nh-1 = H inputs; then one node per operation chunk;
        # then stores.  Per node after the H inputs: the node in word 0's
        # high half (the destination, or the stored value), up to four
        # operand nodes, and the constant bits of each word.
        kinds = ["h"] * nh
        parents = [[] for _ in range(nh)]
        val_node = {i: i for i in range(nh)}   # value id -> node producing it
        dnode, ops, const = [], [], []
        for op in p2.ops:
            if op[0] == "hrr":
                _, d, hi, sym_i, lo = op
                nid = len(kinds)
                kinds.append("hrr")
                a, b = val_node[hi], val_node[lo]
                parents.append([a, b])
                sym, i = sym_i
                dnode.append(nid)
                ops.append((a, b, -1, -1))
                const.append((0, 0, i + (3 if sym == "CD" else 0), 0))
                val_node[d] = nid
            else:
                # rows of more than four terms: the first descriptor sums
                # four, each further one adds 1.0 x the running sum and up to
                # three more
                _, d, terms = op
                prev = None
                rest = list(terms)
                while rest:
                    take = 4 if prev is None else 3
                    chunk, rest = rest[:take], rest[take:]
                    nid = len(kinds)
                    kinds.append("lin")
                    ps = [val_node[s] for _, s in chunk]
                    cfs = [float(cf) for cf, _ in chunk]
                    if prev is not None:
                        ps.append(prev)
                        cfs.append(1.0)
                    parents.append(list(ps))
                    nt = len(ps)
                    cc = [ctab[cf] for cf in cfs] + [0] * (4 - nt)
                    dnode.append(nid)
                    ops.append(tuple(ps) + (-1,) * (4 - nt))
                    const.append((1 | (nt << 2), 0, 0, cc[0] | (cc[1] << 8) | (cc[2] << 16) | (cc[3] << 24)))
                    prev = nid
                val_node[d] = prev
        store_first = len(kinds)
        for k, v in enumerate(p2.outputs):
            kinds.append("store")
            parents.append([val_node[v]])
            i = np.unravel_index(k, p2.out_dims)
            dnode.append(val_node[v])
            ops.append((-1, -1, -1, -1))
            const.append((2, k, int(i[0]) | (int(i[1]) << 8) | (int(i[2]) << 16) | (int(i[3]) << 24), 0))
        n2 = len(kinds)
        self.n2w = n2 - nh                     # scheduled Phase-2 nodes (work ids v - nh)
        prio = np.arange(n2, dtype=np.int64)
        # stores go right after their value: priority of the producer
        for nid in range(store_first, n2):
            prio[nid] = parents[nid][0]
        self.prio2 = prio[nh:].tolist()
        # H inputs are not scheduled (they are read in place)
        par_w = [[p - nh for p in parents[v] if p >= nh] for v in range(nh, n2)]
        self.par2 = par_w
        self.cons2, self.npar2 = _consumer_lists(par_w, self.n2w)
        self.needs2 = np.array([k in ("hrr", "lin") for k in kinds[nh:]], dtype=bool)
        self.dnode2 = np.array(dnode, dtype=np.int64).reshape(-1)
        self.ops2 = np.array(ops, dtype=np.int64).reshape(-1, 4)
        self.const2 = np.array(const, dtype=np.int64).reshape(-1, 4)
        # shape of a Phase-2 node: kind (HRR, linear combination, store),
        # then number of terms
        self.shape2 = ((self.const2[:, 0] & 3) * 8 + ((self.const2[:, 0] >> 2) & 7)).astype(np.int64)


def _static(prog):
    st = getattr(prog, "_coop_static", None)
    if st is None:
        st = _Static(prog)
        prog._coop_static = st
        prog._coop_width = {}
    return st


def release(prog):
    """Drop the cooperative-form caches held on a class program."""
    for name in ("_coop_static", "_coop_width"):
        prog.__dict__.pop(name, None)


def _p1_waves(prog, width, lag):
    st = _static(prog)
    key = ("w1", width, lag)
    if key not in prog._coop_width:
        waves1 = _waves(st.cons1, list(st.npar1), st.prio1, width, lag)
        prog._coop_width[key] = (waves1,) + _lifetimes(st.par1, waves1)
    return prog._coop_width[key]


def _p2_waves(prog, width, lag):
    st = _static(prog)
    key = ("w2", width, lag)
    if key not in prog._coop_width:
        waves2 = _waves(st.cons2, list(st.npar2), st.prio2, width, lag)
        prog._coop_width[key] = (waves2,) + _lifetimes(st.par2, waves2)
    return prog._coop_width[key]


def _p1_rows(st, slot1):
    src = st.src1
    sl = np.where(src >= 0, slot1[np.maximum(src, 0)], 0)
    rows1 = np.empty((st.n1, 4), dtype=np.int64)
    rows1[:, 0] = np.where(st.consumed, slot1, 0xFFFF) | st.hword
    rows1[:, 1] = sl[:, 0] | (sl[:, 1] << 16)
    rows1[:, 2] = sl[:, 2] | (sl[:, 3] << 16)
    rows1[:, 3] = sl[:, 4] | (st.meta1 << 16)
    return rows1


def _p2_rows(st, slot2):
    nh = st.nh
    # operand id of a node: H index, or nh + its value slot
    oid = np.concatenate([np.arange(nh, dtype=np.int64), nh + slot2])

    def ids(nodes):
        return np.where(nodes >= 0, oid[np.maximum(nodes, 0)], 0)

    o = ids(st.ops2)
    c = st.const2
    rows2 = np.empty((st.n2w, 4), dtype=np.int64)
    rows2[:, 0] = c[:, 0] | (ids(st.dnode2) << 16)
    rows2[:, 1] = c[:, 1] | o[:, 0] | (o[:, 1] << 16)
    rows2[:, 2] = c[:, 2] | o[:, 2] | (o[:, 3] << 16)
    rows2[:, 3] = c[:, 3]
    return rows2


def _p1_form(prog, width, lag=1):
    """Phase-1 waves, slots and descriptor rows for waves of up to ``width``
    nodes and parents at least ``lag`` waves back (cached per program, width
    and lag: shapes of equal width share them)."""
    st = _static(prog)
    key = (1, width, lag)
    cached = prog._coop_width.get(key)
    if cached is not None:
        return cached
    waves1, wave_of, last = _p1_waves(prog, width, lag)
    slot1, nslot1 = _allocate(wave_of, last, st.consumed, [v for w in waves1 for v in w], lag=lag)
    form = (waves1, _p1_rows(st, slot1), int(nslot1))
    prog._coop_width[key] = form
    return form


def _p2_form(prog, width, lag=1):
    """Phase-2 waves, slots and descriptor rows (as _p1_form)."""
    st = _static(prog)
    key = (2, width, lag)
    cached = prog._coop_width.get(key)
    if cached is not None:
        return cached
    waves2, wave_of2, last2 = _p2_waves(prog, width, lag)
    slot2, nslot2 = _allocate(wave_of2, last2, st.needs2, [v for w in waves2 for v in w], lag=lag)
    form = (waves2, _p2_rows(st, slot2), int(nslot2))
    prog._coop_width[key] = form
    return form


def _positions(waves, T, ilp, shape):
    """Where _pack puts each node: (global step, lane, node slot of the lane)
    for every node of the waves (-1 elsewhere)."""
    W = ilp * T
    n = int(shape.shape[0])
    step = np.full(n, -1, dtype=np.int64)
    lane = np.full(n, -1, dtype=np.int64)
    u = np.full(n, -1, dtype=np.int64)
    if not len(waves):
        return step, lane, u
    sizes = np.array([len(w) for w in waves], dtype=np.int64)
    steps = (sizes + W - 1) // W
    idx = np.concatenate([np.asarray(w, dtype=np.int64) for w in waves])
    wave_id = np.repeat(np.arange(len(waves)), sizes)
    idx = idx[np.lexsort((np.arange(idx.size), shape[idx], wave_id))]
    k = np.arange(idx.size) - np.repeat(np.cumsum(sizes) - sizes, sizes)
    s, r = np.divmod(k, W)
    step[idx] = np.repeat(np.cumsum(steps) - steps, sizes) + s
    lane[idx] = r % T
    u[idx] = r // T
    return step, lane, u


def _group_key(step, lane, u, k, T, ilp):
    """Access group of a half-warp instruction: operand position k (0-4
    loads, 5 the result store) of node slot u in one half of one warp in
    one step."""
    return (((step * (T // 32) + lane // 32) * 2 + (lane % 32) // 16) * ilp + u) * 6 + k


def _groups_by_value(n, pairs):
    """pairs: (value, group) arrays -> groups[value] (sorted, distinct)."""
    v, g = pairs
    groups = [np.empty(0, dtype=np.int64)] * n
    if v.size == 0:
        return groups
    o = np.lexsort((g, v))
    v, g = v[o], g[o]
    keep = np.ones(v.size, dtype=bool)
    keep[1:] = (v[1:] != v[:-1]) | (g[1:] != g[:-1])
    v, g = v[keep], g[keep]
    cuts = np.flatnonzero(np.diff(v)) + 1
    for vv, gg in zip(np.split(v, cuts), np.split(g, cuts)):
        groups[int(vv[0])] = gg
    return groups


def _p1_banked(prog, width, lag, T, ilp):
    """Phase-1 form with bank-aware slots for teams of T lanes x ilp."""
    st = _static(prog)
    waves1, wave_of, last = _p1_waves(prog, width, lag)
    step, lane, u = _positions(waves1, T, ilp, st.shape1)
    vs, gs = [], []
    node = np.arange(st.n1, dtype=np.int64)
    live = st.consumed
    vs.append(node[live])
    gs.append(_group_key(step[live], lane[live], u[live], 5, T, ilp))
    for k in range(5):
        p = st.src1[:, k]
        m = p >= 0
        vs.append(p[m])
        gs.append(_group_key(step[m], lane[m], u[m], k, T, ilp))
    groups = _groups_by_value(st.n1, (np.concatenate(vs), np.concatenate(gs)))
    slot1, nslot1 = _allocate_banked(wave_of, last, st.consumed, [v for w in waves1 for v in w], groups, lag=lag)
    return waves1, _p1_rows(st, slot1), int(nslot1)


def _p2_banked(prog, width, lag, T, ilp, h_shared):
    """Phase-2 form with bank-aware slots; with h_shared the accumulators
    an instruction reads sit in the same shared memory ([H | slots])."""
    st = _static(prog)
    nh = st.nh
    waves2, wave_of2, last2 = _p2_waves(prog, width, lag)
    step, lane, u = _positions(waves2, T, ilp, st.shape2)
    kind = st.const2[:, 0] & 3
    w = np.arange(st.n2w, dtype=np.int64)
    vs, gs, fixed = [], [], []
    m = st.needs2
    vs.append(w[m])
    gs.append(_group_key(step[m], lane[m], u[m], 5, T, ilp))
    reads = [(st.ops2[:, k], kind != 2, k) for k in range(4)] + [(st.dnode2, kind == 2, 4)]
    for p, sel, k in reads:
        mv = sel & (p >= nh)
        vs.append(p[mv] - nh)
        gs.append(_group_key(step[mv], lane[mv], u[mv], k, T, ilp))
        if h_shared:
            mh = sel & (p >= 0) & (p < nh)
            fixed.append(np.stack([_group_key(step[mh], lane[mh], u[mh], k, T, ilp), (p[mh] - nh) % NBANK], 1))
    groups = _groups_by_value(st.n2w, (np.concatenate(vs), np.concatenate(gs)))
    fx = np.concatenate(fixed) if fixed else None
    slot2, nslot2 = _allocate_banked(wave_of2, last2, st.needs2, [v for wv in waves2 for v in wv], groups,
                                     fixed=fx, lag=lag)
    return waves2, _p2_rows(st, slot2), int(nslot2)


def _width_form(prog, width, lag=1):
    """Both phases' forms for one wave width."""
    return _p1_form(prog, width, lag) + _p2_form(prog, width, lag)


def build(prog, T=128, ilp=ILP, wave_steps=1, lag=1, wave_steps2=None, banked=False, h_shared=True):
    """CoopProgram of a class program for teams of T lanes taking ilp nodes
    per step; a wave (the nodes between two team barriers) holds up to
    wave_steps steps of mutually independent nodes in Phase 1 and
    wave_steps2 (default: wave_steps) in Phase 2.  lag 2: split barriers
    (teams of 64 lanes or more), parents at least two waves back."""
    if lag == 2 and T < 64:
        raise ValueError("split barriers need teams of 64 lanes or more")
    st = _static(prog)
    k2 = wave_steps if wave_steps2 is None else wave_steps2
    if banked:
        # bank-aware slots for this team shape (the slot counts are the same)
        waves1, rows1, nslot1 = _p1_banked(prog, ilp * T * wave_steps, lag, T, ilp)
        waves2, rows2, nslot2 = _p2_banked(prog, ilp * T * k2, lag, T, ilp, h_shared)
    else:
        waves1, rows1, nslot1 = _p1_form(prog, ilp * T * wave_steps, lag)
        waves2, rows2, nslot2 = _p2_form(prog, ilp * T * k2, lag)
    ph1, steps1 = _pack(waves1, rows1, T, NOP1, ilp, st.shape1)
    ph2, steps2 = _pack(waves2, rows2, T, NOP2, ilp, st.shape2)
    nh = st.nh
    nslot = max(nslot1, nslot2)
    if nslot >= 0xFFFF or nh + nslot > MAX_ID:
        raise ValueError("class {} needs {} ids".format(prog.ls, nh + nslot))
    eff1 = st.n1 / max(1, int(steps1.sum()) * T * ilp)
    eff2 = st.n2w / max(1, int(steps2.sum()) * T * ilp)
    assert ph1.shape[0] == (int(steps1.sum()) + PREFETCH_STEPS) * T * ilp
    cp = CoopProgram(T, ilp, ph1, steps1, ph2, steps2, nh, nslot, prog.L, tuple(prog.p2.out_dims), eff1, eff2,
                     lag)
    cp.wave_steps, cp.wave_steps2 = wave_steps, k2
    return cp


def _half_warp_wavefronts(ids, mask):
    """Wavefronts of 64-bit shared accesses: ids, mask [..., 32 lanes] per
    warp instruction; each half-warp costs the most distinct words it finds
    in one of the 16 bank pairs (a repeated word is a broadcast)."""
    x = np.where(mask, ids, -1).reshape(-1, 16)
    x = x[(x >= 0).any(axis=1)]
    if x.size == 0:
        return 0, 0
    x = np.sort(x, axis=1)
    dup = np.zeros_like(x, dtype=bool)
    dup[:, 1:] = x[:, 1:] == x[:, :-1]
    ok = (x >= 0) & ~dup
    r, c = np.nonzero(ok)
    cnt = np.zeros((x.shape[0], NBANK), dtype=np.int64)
    np.add.at(cnt, (r, x[r, c] % NBANK), 1)
    return int(cnt.max(axis=1).sum()), int(x.shape[0])


def shared_wavefronts(cp, h_shared=False):
    """Modelled shared-memory wavefronts of a cooperative program's value-slot
    accesses and the conflict-free count: (Phase-1 wavefronts, Phase-1
    ideal, Phase-2 wavefronts, Phase-2 ideal); Phase 1 per primitive
    quartet, Phase 2 per shell quartet.  Each operand position of a step's
    node slot is one warp instruction (loads a..e and the result store in
    Phase 1; the four operands, the stored value and the result in Phase
    2); with h_shared the accumulators Phase 2 reads count as shared
    operands at their own banks."""
    W = cp.T * cp.ilp
    warps = cp.T // 32

    def slots(ph, steps):
        n = int(np.sum(steps))
        d = ph[: n * W].astype(np.int64).reshape(n, warps, 32, cp.ilp, 4)
        return np.moveaxis(d, 3, 2)          # [step, warp, ilp, lane, word]

    d = slots(cp.ph1, cp.steps1)
    meta = d[..., 3] >> 16
    term = (meta & 0xC000) == 0
    t2 = term & (((meta >> 4) & 31) > 0)
    t3 = term & (((meta >> 9) & 15) > 0)
    dst = d[..., 0] & 0xFFFF
    acc = [(d[..., 1] & 0xFFFF, term), (d[..., 1] >> 16, term), (d[..., 2] & 0xFFFF, t2), (d[..., 2] >> 16, t2),
           (d[..., 3] & 0xFFFF, t3), (dst, ((meta & 0x8000) == 0) & (dst != 0xFFFF))]
    w1 = [_half_warp_wavefronts(a, m) for a, m in acc]
    d = slots(cp.ph2, cp.steps2)
    nh = cp.nh
    kind = d[..., 0] & 3
    nt = (d[..., 0] >> 2) & 7
    lo = 0 if h_shared else nh              # lowest operand id in shared memory
    ops = [(d[..., 1] & 0xFFFF, (kind == 0) | (kind == 1)), (d[..., 1] >> 16, (kind == 0) | ((kind == 1) & (nt > 1))),
           (d[..., 2] & 0xFFFF, (kind == 1) & (nt > 2)), (d[..., 2] >> 16, (kind == 1) & (nt > 3)),
           (d[..., 0] >> 16, kind == 2), (d[..., 0] >> 16, (kind <= 1))]
    w2 = [_half_warp_wavefronts(a, m & (a >= lo)) for a, m in ops]
    return (sum(a for a, _ in w1), sum(b for _, b in w1), sum(a for a, _ in w2), sum(b for _, b in w2))


def fp64_issue(cp):
    """FP64 warp-instructions the cooperative executor issues for a program:
    (Phase 1 per primitive quartet, Phase 2 per shell quartet).  A warp
    issues an instruction whenever one of its 32 lanes needs it (a
    predicated-off lane still takes the issue slot): per descriptor slot, a
    Phase-1 node costs a multiply and an FMA, two more FMAs when it has the
    second Obara-Saika term and one more for the cross term; an HRR step one
    FMA; a linear combination of n terms a multiply and n - 1 FMAs.  H
    updates (atomic reductions in global memory) and stores of a quartet's
    first part issue none.  With a class's algorithmic flops this gives the
    fraction of the FP64 FMA rate the program could reach if the pipe never
    waited."""
    W = cp.T * cp.ilp
    warps = cp.T // 32

    def slots(ph, steps):
        n = int(np.sum(steps))
        return ph[: n * W].astype(np.int64).reshape(n, warps, 32, cp.ilp, 4)

    def any_lane(m):
        return m.any(axis=2).astype(np.int64)

    d = slots(cp.ph1, cp.steps1)
    meta = d[..., 3] >> 16
    term = (meta & 0xC000) == 0
    i1 = (2 * any_lane(term) + 2 * any_lane(term & (((meta >> 4) & 31) > 0))
          + any_lane(term & (((meta >> 9) & 15) > 0)))
    d = slots(cp.ph2, cp.steps2)
    kind = d[..., 0] & 3
    nt = (d[..., 0] >> 2) & 7
    lin = kind == 1
    i2 = (any_lane(kind == 0) + any_lane(lin) + any_lane(lin & (nt > 1)) + any_lane(lin & (nt > 2))
          + any_lane(lin & (nt > 3)))
    return int(i1.sum()), int(i2.sum())


def fp64_balance(cp):
    """How evenly a team's Phase-1 FP64 work is spread over the SM's four
    sub-partitions within each wave (warp w of a team runs on sub-partition
    w mod 4; the waves end at a barrier, so a wave lasts as long as its
    busiest sub-partition): sum over waves of the FP64 warp-instructions
    divided by sum over waves of 4 x the busiest sub-partition's share.  1.0
    is perfect balance; meaningful for teams of 128 lanes or more, which
    hold warps on all four sub-partitions."""
    W = cp.T * cp.ilp
    warps = cp.T // 32
    n = int(np.sum(cp.steps1))
    d = cp.ph1[: n * W].astype(np.int64).reshape(n, warps, 32, cp.ilp, 4)
    meta = d[..., 3] >> 16
    term = (meta & 0xC000) == 0

    def any_lane(m):
        return m.any(axis=2).astype(np.int64)

    per = (2 * any_lane(term) + 2 * any_lane(term & (((meta >> 4) & 31) > 0))
           + any_lane(term & (((meta >> 9) & 15) > 0))).sum(axis=2)  # [step, warp]
    bounds = np.concatenate([[0], np.cumsum(cp.steps1.astype(np.int64))])
    total = busiest = 0
    for w in range(len(cp.steps1)):
        per_warp = per[bounds[w]:bounds[w + 1]].sum(axis=0)
        sub = np.bincount(np.arange(warps) % 4, weights=per_warp, minlength=4)
        total += sub.sum()
        busiest += 4 * sub.max()
    return float(total / busiest) if busiest else 1.0


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


# Split-barrier forms (waves scheduled with parents two waves back, so a lane
# may start a wave while others finish the previous one) were measured on
# GB300 against full barriers and lost 2-5% on (dd|dd), (ff|ff) and (gg|gg):
# their extra steps cost more than the barrier drains they save.  The build
# takes full-barrier forms; the schedule stays available (split=True).
SPLIT_BARRIERS = False
WIDE_SHAPES = ((256, 2), (256, 4))
# sixteen warps on one live set: 512 lanes, two nodes per lane (the register
# file holds 128 registers for each of 512 threads)
WIDEST_SHAPE = (512, 2)
# nodes in a multi-step wave of a 512-lane team: four steps.  Measured on
# (gg|gg) against two-step waves (27 instead of 44 Phase-1 barriers per
# primitive quartet, 25,523 instead of 22,760 slots, still one team and 16
# warps per SM): 0.653 -> 0.672 of the FP64 rate on the sweep, 0.647 ->
# 0.663 at K = 6, 0.466 -> 0.485 at K = 1.
WAVE_NODES_MAX = 4096


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
    in a wave (512 lanes x 2 nodes x 4 steps); narrower teams keep one step per
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


PHASE2_STEPS = (8, 4, 2)  # candidate steps per Phase-2 wave
PHASE2_SMEM_GROWTH = 12 * 1024  # shared memory per SM a wider Phase 2 may add


def _runtime_layout(cp, rows):
    """(resident warps, shared memory per SM) of a shape as the runtime lays
    it out: teams of up to 128 lanes share 128-thread blocks, wider teams
    fill a block; H goes in shared memory when that keeps as many warps;
    at most 512 threads per SM (256 for four nodes per lane)."""
    elem, reserve = 8, 1024
    max_threads = 256 if cp.ilp == 4 else 512
    best = (-1, 0)
    for h_in in (1, 0):
        tpb_max = max(1, 128 // cp.T)
        tpb = tpb_max
        while tpb >= 1:
            per_team = rows * (ROW_BYTES // 8) + cp.nslot + (cp.nh if h_in else 0)
            bsm = (per_team * tpb * elem + 15) // 16 * 16
            if bsm <= 227 * 1024:
                bps = min(max_threads // (tpb * cp.T), max(1, SMEM_PER_SM // (bsm + reserve)))
                warps = bps * tpb * cp.T // 32
                if bps >= 1 and warps > best[0]:
                    best = (warps, bps * bsm)
            tpb //= 2
    return best


def _wide_phase2(prog, cp, rows):
    """Phase 2 runs once per shell quartet (the HRR and the transform), after
    the contraction: with few primitive quartets per shell quartet it weighs
    as much as Phase 1, and its barriers more (the (gg|gg) Phase-2 graph
    spreads over 159 two-step waves).  Its live set is smaller than Phase
    1's, so wider Phase-2 waves often cost no value slots at all ((gg|gg):
    four-step waves need 18,586 slots against Phase 1's 22,760).  Take the
    widest of 8, 4 and 2 steps per Phase-2 wave that keeps the teams per SM;
    Phase 1 keeps its form.  A wider Phase 2 must keep the warps the
    runtime makes resident and add at most PHASE2_SMEM_GROWTH of shared
    memory per SM: the rest of the SM's 256 KB is L1, which holds the
    descriptor stream.  Measured with eight-step Phase-2 waves wherever the
    generator's team count held: (ff|ff) grew from 4,965 to 6,766 slots,
    which cut the runtime's warps per SM from 16 to 12 and cost 5% at K = 3
    and 6; (gg|gg) grew 24 KB per SM at 16 warps and lost 1% at K = 6 (8%
    gained at K = 1); (dd|dd) grew 10 KB at 16 warps and gained 18% at
    K = 1 and 2% at K = 3 and 6."""
    if cp is None:
        return cp
    k1 = getattr(cp, "wave_steps", 1)
    k0 = getattr(cp, "wave_steps2", k1)
    warps0, smem0 = _runtime_layout(cp, rows)
    for k in PHASE2_STEPS:
        if k <= k0:
            break
        ck = build(prog, cp.T, cp.ilp, k1, cp.lag, wave_steps2=k)
        if _score(ck, rows) is None:
            continue
        warps, smem = _runtime_layout(ck, rows)
        if warps >= warps0 and smem <= smem0 + PHASE2_SMEM_GROWTH:
            return ck
    return cp


# split barriers cost no drain at a wave's end but put a node's parents at
# least two waves back, which can stretch a narrow graph: they are taken when
# the steps they need stay within this factor of the full-barrier form's
SPLIT_STEP_RATIO = 1.15


def _split_barriers(prog, cp, rows):
    """The same team shape with split barriers (one step per wave, parents at
    least two waves back, slots released a wave later), when it keeps the
    teams per SM and its steps stay within SPLIT_STEP_RATIO of the
    full-barrier form's, else None.  Teams of one warp keep full barriers
    (a warp-synchronous point costs no drain)."""
    if cp is None or cp.T < 64:
        return None
    ck = build(prog, cp.T, cp.ilp, 1, lag=2)
    if _score(ck, rows) is None or _teams_per_sm(ck, rows) < _teams_per_sm(cp, rows):
        return None
    steps = lambda c: int(c.steps1.sum()) + int(c.steps2.sum()) / 8.0
    return ck if steps(ck) <= SPLIT_STEP_RATIO * steps(cp) else None


BANKED = True  # bank-aware value slots in the shipped programs


def _banked(prog, cp, rows):
    """The same shape with bank-aware slots (same slot count).  Phase 2
    counts the accumulators it reads as shared-memory operands when H fits
    in shared memory beside the slots (the runtime's preference)."""
    if cp is None or not BANKED:
        return cp
    h_shared = cp.nslot * 8 + rows * ROW_BYTES + cp.nh * 8 <= 227 * 1024
    k1 = getattr(cp, "wave_steps", 1)
    return build(prog, cp.T, cp.ilp, k1, cp.lag, wave_steps2=getattr(cp, "wave_steps2", k1), banked=True,
                 h_shared=h_shared)


def shape_key(cp):
    """What tells two cooperative programs of one class apart: team size,
    nodes per lane, steps per Phase-1 and per Phase-2 wave."""
    k1 = getattr(cp, "wave_steps", 1)
    return (cp.T, cp.ilp, k1, getattr(cp, "wave_steps2", k1))


def choose_both(prog, shapes=SHAPES, split=None, wide2=True, alts=0):
    """(deep, shallow): the best (team size, nodes per lane) shape when a
    team holds DEEP_ROWS coefficient rows, and when it holds SHALLOW_ROWS
    (shallow contractions: fewer rows leave shared memory for more teams).
    Classes whose 128-lane team is alone on an SM also try one 256-lane team
    (eight warps on the same shared-memory live set), and those whose
    256-lane team is alone even with H in global memory one 512-lane team
    (sixteen warps).  With alts > 0 also a list of up to `alts` other
    shapes, the next best by score with their wave depths chosen the same
    way: candidates an autotuner can time against the static choice."""
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
        cp = _wide_waves(prog, built[max(scored)[1]], rows) if scored else None
        if SPLIT_BARRIERS if split is None else split:
            cp = _split_barriers(prog, cp, rows) or cp
        elif wide2:
            cp = _wide_phase2(prog, cp, rows)
        out.append(cp)
    if alts > 0:
        taken = {shape_key(cp) for cp in out if cp is not None}
        scored = sorted(((sc, k) for k, cp in enumerate(built) for sc in [_score(cp, DEEP_ROWS)] if sc is not None),
                        reverse=True)
        extra = []
        for _, k in scored:
            if len(extra) >= alts:
                break
            cp = _wide_waves(prog, built[k], DEEP_ROWS)
            if wide2:
                cp = _wide_phase2(prog, cp, DEEP_ROWS)
            if shape_key(cp) not in taken:
                taken.add(shape_key(cp))
                extra.append(cp)
        out.append(extra)
    out[0] = _banked(prog, out[0], DEEP_ROWS)
    out[1] = (out[0] if out[1] is not None and out[0] is not None and shape_key(out[1]) == shape_key(out[0])
              else _banked(prog, out[1], SHALLOW_ROWS))
    if alts > 0:
        out[2] = [_banked(prog, cp, DEEP_ROWS) for cp in out[2]]
    release(prog)
    return tuple(out)


def choose(prog, shapes=SHAPES):
    """The best shape for deep contractions (see choose_both)."""
    return choose_both(prog, shapes)[0]
