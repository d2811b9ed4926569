"""Phase 1 of the HGP scheme: the Obara-Saika vertical recurrence graph.

A node is [e0|f0]^(m) (FusionRCG Sec. II-A, Eq. 2).  Each non-base node is
reduced along one axis of the bra (e) or the ket (f):

  bra, axis i:  [e|f]^m = PA_i [e-1i|f]^m + WP_i [e-1i|f]^(m+1)
                + (e_i-1)/(2 zeta) ([e-2i|f]^m - rho/zeta [e-2i|f]^(m+1))
                + f_i/(2(zeta+eta)) [e-1i|f-1i]^(m+1)
  ket, axis i:  [e|f]^m = QC_i [e|f-1i]^m + WQ_i [e|f-1i]^(m+1)
                + (f_i-1)/(2 eta) ([e|f-2i]^m - rho/eta [e|f-2i]^(m+1))
                + e_i/(2(zeta+eta)) [e-1i|f-1i]^(m+1)

(the ket form is the mirror image of Eq. 2, which the paper does not print).
Base nodes [00|00]^(m) come from the Boys function.

Axis rules (which axis reduces a node):
  "prose"   consumer first: any f_i > 0 -> ket, largest such i (z, y, x);
            else bra, largest i with e_i > 0  (Sec. III-A text);
  "literal" Algorithm 1 as printed: scan i = 0, 1, 2, the last i with
            c_i > 0 (ket) or a_i > 0 (bra) wins, ket preferred at equal i;
  "common"  the conventional order of the ablation: bra first, x -> y -> z.

Scheduling: "dsa" is the greedy list scheduler of Eq. 7 (static score
sum_{w in Reach(v)} out(w) - in(w), Reach reflexive); "level" is a plain
safe order (by total angular momentum, then m), the ablation's "No DSA".
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass, field

import numpy as np

from . import cart

AXIS_RULES = ("prose", "literal", "common")
SCHEDULES = ("dsa", "level")


def choose_axis(e, f, rule):
    """(side, axis) for node (e, f): side 0 = bra, 1 = ket."""
    if rule == "prose":
        for i in (2, 1, 0):
            if f[i] > 0:
                return 1, i
        for i in (2, 1, 0):
            if e[i] > 0:
                return 0, i
    elif rule == "literal":
        pick = None
        for i in (0, 1, 2):
            if f[i] > 0:
                pick = (1, i)
            elif e[i] > 0:
                pick = (0, i)
        return pick
    elif rule == "common":
        for i in (0, 1, 2):
            if e[i] > 0:
                return 0, i
        for i in (0, 1, 2):
            if f[i] > 0:
                return 1, i
    else:
        raise ValueError(rule)
    return None


@dataclass
class VrrGraph:
    la: int
    lb: int
    lc: int
    ld: int
    rule: str
    keys: list = field(default_factory=list)      # node id -> (e, f, m)
    terms: list = field(default_factory=list)     # node id -> [(coef, parent id)]
    side: list = field(default_factory=list)      # node id -> -1 base, 0 bra, 1 ket
    target: dict = field(default_factory=dict)    # node id -> H index
    ids: dict = field(default_factory=dict)

    @property
    def L(self):
        return self.la + self.lb + self.lc + self.ld

    def __len__(self):
        return len(self.keys)


def h_layout(la, lb, lc, ld):
    """Contracted accumulator layout H[ie][jf]: e over degrees la..la+lb, f over
    lc..lc+ld, each in Cartesian order."""
    E = cart.range_tuples(la, la + lb)
    F = cart.range_tuples(lc, lc + ld)
    return E, F


def build(la, lb, lc, ld, rule="prose") -> VrrGraph:
    g = VrrGraph(la, lb, lc, ld, rule)
    z3 = (0, 0, 0)

    def node(e, f, m):
        key = (e, f, m)
        if key in g.ids:
            return g.ids[key]
        if e == z3 and f == z3:
            terms, side = [], -1
        else:
            side, i = choose_axis(e, f, rule)
            terms = []
            if side == 0:
                e1 = cart.sub(e, i)
                terms.append((("PA", i), node(e1, f, m)))
                terms.append((("WP", i), node(e1, f, m + 1)))
                if e[i] >= 2:
                    e2 = cart.sub(e, i, 2)
                    terms.append((("c1z", e[i] - 1), node(e2, f, m)))
                    terms.append((("c2z", e[i] - 1), node(e2, f, m + 1)))
                if f[i] >= 1:
                    terms.append((("c3", f[i]), node(e1, cart.sub(f, i), m + 1)))
            else:
                f1 = cart.sub(f, i)
                terms.append((("QC", i), node(e, f1, m)))
                terms.append((("WQ", i), node(e, f1, m + 1)))
                if f[i] >= 2:
                    f2 = cart.sub(f, i, 2)
                    terms.append((("c1e", f[i] - 1), node(e, f2, m)))
                    terms.append((("c2e", f[i] - 1), node(e, f2, m + 1)))
                if e[i] >= 1:
                    terms.append((("c3", e[i]), node(cart.sub(e, i), f1, m + 1)))
        nid = len(g.keys)
        g.ids[key] = nid
        g.keys.append(key)
        g.terms.append(terms)
        g.side.append(side)
        return nid

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 20000))
    try:
        E, F = h_layout(la, lb, lc, ld)
        nf = len(F)
        for ie, e in enumerate(E):
            for jf, f in enumerate(F):
                g.target[node(e, f, 0)] = ie * nf + jf
    finally:
        sys.setrecursionlimit(old)
    return g


# ---------------------------------------------------------------------------
# scheduling
# ---------------------------------------------------------------------------
def _consumers(g):
    cons = [[] for _ in range(len(g))]
    for v, ts in enumerate(g.terms):
        for _, p in ts:
            cons[p].append(v)
    return cons


def dsa_scores(g, window: int = 8192) -> np.ndarray:
    """score(v) = sum over w in Reach(v) (v and everything downstream of it)
    of out(w) - in(w), computed exactly with bitsets over windows of w."""
    n = len(g)
    cons = _consumers(g)
    outd = np.array([len(set(c)) for c in cons], dtype=np.int64)
    ind = np.array([len(set(p for _, p in ts)) for ts in g.terms], dtype=np.int64)
    d = outd - ind
    # reverse topological order: node ids are created parents-first, so
    # descending id is a valid reverse topological order.  Group by depth so
    # that numpy can OR whole levels at once.
    depth = np.zeros(n, dtype=np.int64)  # longest path to a sink
    for v in range(n - 1, -1, -1):
        if cons[v]:
            depth[v] = 1 + max(depth[c] for c in cons[v])
    maxc = max((len(c) for c in cons), default=0)
    cmat = np.full((n, max(maxc, 1)), n, dtype=np.int64)  # n = no consumer
    for v, c in enumerate(cons):
        cmat[v, :len(c)] = c
    levels = [np.nonzero(depth == k)[0] for k in range(int(depth.max()) + 1 if n else 0)]
    score = np.zeros(n, dtype=np.int64)
    for w0 in range(0, n, window):
        w1 = min(n, w0 + window)
        # bit position of each node of the window: grouped by d(w), every
        # group starting on a word, so that one popcount per word weighted
        # by its group's d gives the sum
        dw = d[w0:w1]
        order = np.argsort(dw, kind="stable")
        vals, counts = np.unique(dw, return_counts=True)
        gwords = (counts + 63) // 64
        start = np.repeat((np.cumsum(gwords) - gwords) * 64, counts)
        pos = np.empty(w1 - w0, dtype=np.int64)
        pos[order] = start + np.arange(w1 - w0) - np.repeat(np.cumsum(counts) - counts, counts)
        words = int(gwords.sum())
        # rows 0..w1-1, and row w1 (zero) for consumers at or beyond w1:
        # a node at or beyond w1 reaches only later nodes, none in the window
        bits = np.zeros((w1 + 1, words), dtype=np.uint64)
        own = np.arange(w0, w1)
        bits[own, pos // 64] |= np.uint64(1) << (pos % 64).astype(np.uint64)
        for lev in levels:
            lev = lev[: np.searchsorted(lev, w1)]
            if lev.size == 0:
                continue
            ch = np.minimum(cmat[lev], w1)
            acc = bits[lev]
            for k in range(ch.shape[1]):
                acc |= bits[ch[:, k]]
            bits[lev] = acc
        weight = np.repeat(vals, gwords)
        score[:w1] += np.bitwise_count(bits[:w1]).astype(np.int64) @ weight
    return score


def schedule(g, how="dsa"):
    n = len(g)
    if how == "level":
        def key(v):
            e, f, m = g.keys[v]
            return (sum(e) + sum(f), -m, e, f)
        return sorted(range(n), key=key)
    if how != "dsa":
        raise ValueError(how)
    score = dsa_scores(g)
    cons = _consumers(g)
    npar = [len(set(p for _, p in ts)) for ts in g.terms]
    left = list(npar)
    ready = [(-int(score[v]), v) for v in range(n) if npar[v] == 0]
    heapq.heapify(ready)
    order = []
    for _ in range(n):
        _, v = heapq.heappop(ready)
        order.append(v)
        for c in set(cons[v]):
            left[c] -= 1
            if left[c] == 0:
                heapq.heappush(ready, (-int(score[c]), c))
    assert len(order) == n
    return order


def check_topological(g, order) -> bool:
    pos = {v: i for i, v in enumerate(order)}
    if len(pos) != len(g):
        return False
    return all(pos[p] < pos[v] for v, ts in enumerate(g.terms) for _, p in ts)


def lifetimes(g, order):
    """Birth (step of definition) and death (step of last use; birth if unused)
    for every node under ``order``."""
    pos = np.empty(len(g), dtype=np.int64)
    pos[np.array(order, dtype=np.int64)] = np.arange(len(order))
    death = pos.copy()
    for v, ts in enumerate(g.terms):
        for _, p in ts:
            death[p] = max(death[p], pos[v])
    return pos, death


def peak_live(g, order) -> int:
    """Eq. 4 from lifetimes: at step t, live = values with birth <= t <= death
    (a value is held through the step of its last use)."""
    birth, death = lifetimes(g, order)
    n = len(order)
    delta = np.zeros(n + 1, dtype=np.int64)
    np.add.at(delta, birth, 1)
    np.add.at(delta, death + 1, -1)
    return int(np.cumsum(delta)[:n].max()) if n else 0


def allocate_slots(g, order, reuse_at_last_use=True):
    """Lifetime slot allocation.  A dry run over ``order`` gives every value
    its birth and death step; a linear scan then hands each value the
    lowest-numbered free slot at its birth (for equal-size slots this packs
    to exactly the interval-graph bound, the same count a reverse-time
    best-fit pass reaches).  With ``reuse_at_last_use`` a result may take the
    slot of an operand whose last use is the same step (operands are read
    before the result is written).  Returns (slot per node, number of slots)."""
    birth, death = lifetimes(g, order)
    slot = np.full(len(g), -1, dtype=np.int64)
    free = []
    nslot = 0
    for t, v in enumerate(order):
        dying = [p for p in set(p for _, p in g.terms[v]) if death[p] == t]
        if reuse_at_last_use:
            for p in dying:
                heapq.heappush(free, int(slot[p]))
        if free:
            slot[v] = heapq.heappop(free)
        else:
            slot[v] = nslot
            nslot += 1
        if not reuse_at_last_use:
            for p in dying:
                heapq.heappush(free, int(slot[p]))
        if death[v] == t:  # consumed only by the contraction, at definition
            heapq.heappush(free, int(slot[v]))
    return slot, nslot


def verify_slots(g, order, slot, reuse_at_last_use=True) -> bool:
    """No two values that are live at the same time share a slot."""
    birth, death = lifetimes(g, order)
    owner = {}
    for t, v in enumerate(order):
        s = int(slot[v])
        for p in set(p for _, p in g.terms[v]):
            if owner.get(int(slot[p])) != p:
                return False  # operand was overwritten before this use
        if s in owner and owner[s] is not None:
            prev = owner[s]
            if death[prev] > t or (death[prev] == t and not reuse_at_last_use):
                return False
        owner[s] = v
    return True
