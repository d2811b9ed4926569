"""Binary form of a class program for the program-driven tiers.

The straight-line program of a class (Phase-1 graph in its schedule order,
Phase-2 operations in their liveness-friendly build order, output stores) is
written as fixed 16-byte descriptors that one compiled executor kernel walks.
Every lane of a warp reads the same descriptor, so the walk costs broadcast
loads and a few integer operations per node, which the FP64 pipe hides.

Value slots (16-bit): accumulators H occupy [0, nh); Phase-1 values take
[nh, nh + nslot1) from the lifetime allocator; Phase 2 reuses the whole
space, an accumulator slot becoming free after its last use.

Phase-1 descriptor (uint32 x4):
  w0 = dst | (h + 1) << 16          h = accumulator index, 0 = not a target
  w1 = src0 | src1 << 16
  w2 = src2 | src3 << 16
  w3 = src4 | side << 16 | axis << 18 | k << 20 | k3 << 25 | store << 30
       side 0 bra / 1 ket / 2 base (then k = Boys order m);
       terms: (PA|QC)_axis src0, (WP|WQ)_axis src1,
              k > 0:  c1_k src2, c2_k src3;   k3 > 0: c3_k3 src4
       store = the value is read later (otherwise it only feeds H)
Phase-2 descriptor:
  HRR   w0 = 0 | dst << 16; w1 = hi | lo << 16; w2 = axis (0-2 A-B, 3-5 C-D)
        dst = hi + X_axis * lo
  LIN   w0 = 1 | n << 2 | acc << 5 | dst << 16; w1 = s0 | s1 << 16;
        w2 = s2 | s3 << 16; w3 = c0 | c1 << 8 | c2 << 16 | c3 << 24
        dst = (acc ? dst : 0) + sum_{j<n} coef[c_j] * s_j, n <= 4
  STORE w0 = 2 | src << 16; w1 = output element (canonical row-major);
        w2 = mu | nu << 8 | lam << 16 | sig << 24 (its four component indices)
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache
import heapq

import numpy as np

from . import sph, vrr

MAX_SLOTS = 65535


@lru_cache(maxsize=None)
def coef_table():
    """Distinct transform coefficients of T^(l), l <= 4 (index < 256)."""
    vals = []
    for l in range(5):
        T = sph.matrix(l)
        for x in T[T != 0.0]:
            x = float(x)
            if x not in vals:
                vals.append(x)
    return tuple(vals)


@dataclass
class Encoded:
    ph1: np.ndarray      # uint32 [n1, 4]
    ph2: np.ndarray      # uint32 [n2, 4]
    nh: int
    nslot: int           # total slot space
    kmax: int            # largest k / k3 in Phase 1
    L: int
    out_dims: tuple


def _phase1(prog):
    g = prog.g
    nh = prog.nh
    consumed = set(p for ts in g.terms for _, p in ts)
    rows = np.zeros((len(prog.order), 4), dtype=np.uint32)
    kmax = 0
    for r, v in enumerate(prog.order):
        ts = g.terms[v]
        dst = nh + prog.slot[v]
        h = g.target.get(v)
        w0 = dst | ((h + 1) << 16 if h is not None else 0)
        src = [0] * 5
        side = axis = k = k3 = 0
        if not ts:
            side = 2
            k = g.keys[v][2]
        else:
            for (kind, val), p in ts:
                s = nh + prog.slot[p]
                if kind in ("PA", "QC"):
                    src[0] = s
                    side = 0 if kind == "PA" else 1
                    axis = val
                elif kind in ("WP", "WQ"):
                    src[1] = s
                elif kind in ("c1z", "c1e"):
                    src[2] = s
                    k = val
                elif kind in ("c2z", "c2e"):
                    src[3] = s
                elif kind == "c3":
                    src[4] = s
                    k3 = val
            kmax = max(kmax, k, k3)
        store = 1 if v in consumed else 0
        rows[r, 0] = w0
        rows[r, 1] = src[0] | (src[1] << 16)
        rows[r, 2] = src[2] | (src[3] << 16)
        rows[r, 3] = src[4] | (side << 16) | (axis << 18) | (k << 20) | (k3 << 25) | (store << 30)
    return rows, kmax


def _phase2(prog, first_free):
    """Slot-allocate and encode Phase 2.  Output values are stored by an
    explicit STORE right after they become available and then die."""
    p2 = prog.p2
    nh = prog.nh
    ctab = {c: i for i, c in enumerate(coef_table())}
    # uses of each value: operand reads and output stores
    last_use = {}
    producer = {}
    for t, op in enumerate(p2.ops):
        producer[op[1]] = t
        srcs = [op[2], op[4]] if op[0] == "hrr" else [s for _, s in op[2]]
        for s in srcs:
            last_use[s] = t
    outs_at = {}  # op index -> [(out element, value)], -1 = before any op
    for k, v in enumerate(p2.outputs):
        t = producer.get(v, -1)
        outs_at.setdefault(t, []).append((k, v))
        last_use[v] = max(last_use.get(v, -1), t)
    slot = {i: i for i in range(nh)}
    free = list(range(first_free, MAX_SLOTS))
    heapq.heapify(free)
    used_max = first_free
    rows = []

    def release(v, t):
        if last_use.get(v, -1) <= t and v in slot:
            heapq.heappush(free, slot.pop(v))

    dims = p2.out_dims

    def store(k, v):
        i = np.unravel_index(k, dims)
        rows.append([2 | (slot[v] << 16), k, int(i[0]) | (int(i[1]) << 8) | (int(i[2]) << 16) | (int(i[3]) << 24), 0])

    for k, v in outs_at.get(-1, []):
        store(k, v)
    for v in range(nh):
        release(v, -1)
    for t, op in enumerate(p2.ops):
        srcs = [op[2], op[4]] if op[0] == "hrr" else [s for _, s in op[2]]
        src_slots = [slot[s] for s in srcs]
        d = op[1]
        # the result never shares a slot with an operand: a LIN split over
        # two descriptors reads operands after its first write
        slot[d] = heapq.heappop(free)
        used_max = max(used_max, slot[d] + 1)
        if op[0] == "hrr":
            _, _, _, (sym, i), _ = op
            rows.append([0 | (slot[d] << 16), src_slots[0] | (src_slots[1] << 16), i + (3 if sym == "CD" else 0), 0])
        else:
            terms = list(zip([c for c, _ in op[2]], src_slots))
            for j0 in range(0, len(terms), 4):
                chunk = terms[j0:j0 + 4]
                n = len(chunk)
                ss = [x for _, x in chunk] + [0] * (4 - n)
                cc = [ctab[float(c)] for c, _ in chunk] + [0] * (4 - n)
                rows.append([1 | (n << 2) | ((1 if j0 else 0) << 5) | (slot[d] << 16),
                             ss[0] | (ss[1] << 16), ss[2] | (ss[3] << 16),
                             cc[0] | (cc[1] << 8) | (cc[2] << 16) | (cc[3] << 24)])
        for k, v in outs_at.get(t, []):
            store(k, v)
        for v in set(srcs) | {d}:
            release(v, t)
    return np.array(rows, dtype=np.uint32).reshape(-1, 4), used_max


def encode(prog) -> Encoded:
    ph1, kmax = _phase1(prog)
    nslot1 = prog.nh + prog.nslot
    ph2, used = _phase2(prog, prog.nh)
    nslot = max(nslot1, used)
    if nslot > MAX_SLOTS:
        raise ValueError("class {} needs {} slots".format(prog.ls, nslot))
    return Encoded(ph1, ph2, prog.nh, nslot, kmax, prog.L, tuple(prog.p2.out_dims))
