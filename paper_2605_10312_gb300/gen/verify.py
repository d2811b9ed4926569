"""Static bounds verification of generated class programs.

The program-driven kernels trust their descriptors: a slot, accumulator,
coefficient-row, transform-table or output index is used as it stands,
with no device-side check.  This module proves, on the host and for every
program the build writes, that each such index lies inside the region the
kernel addresses with it:

  team-cooperative programs (coop executor)
    Phase 1: destination slot < nslot (or 0xFFFF: not kept); accumulator
      h - 1 < nh; operand slots < nslot for every term the node evaluates;
      coefficient-row entries inside the 56-entry row: P-A / W-P (side 0) or
      Q-C / W-Q (side 1) with axis < 3, k <= 8, k3 <= 8, Boys order m <= L
      for a base node;
    Phase 2: operand and destination ids < nh + nslot (accumulators, then
      slots), HRR axis < 6, 1..4 terms per linear combination, coefficient
      indexes < the transform table, stores of element k < prod(dims) at
      component indexes that ravel to k;
    layout: descriptor count = (steps + PREFETCH_STEPS) x T x ilp, every
      wave at least one step (a split-barrier program may have empty waves:
      pure synchronisation points), the trailing prefetch steps no-ops;
    hazards: within a wave no slot is both read and written, or written
      twice; with split barriers (lag 2, a lane may run wave w + 1 while
      others still run wave w) neither does any slot between two adjacent
      waves -- nothing wave w + 1 reads or writes is written or read in
      wave w -- so any interleaving of two adjacent waves gives the
      wave-by-wave result; each accumulator has one Phase-1 owner;
  encoded programs (thread-per-quartet executor): the same rules on its
    descriptor form, with one slot space of nslot ids (accumulators first).

verify_coop / verify_encoded return a list of messages (empty: in bounds);
check() raises on the first failing program.
"""
from __future__ import annotations

import numpy as np

from .coop import NOP1, NOP2, PREFETCH_STEPS

ROW_ENTRIES = 56      # coefficient row of one primitive quartet (coop executor)
MAX_K = 8             # largest k / k3 of an Obara-Saika term


def _bad(mask, what, out):
    n = int(np.count_nonzero(mask))
    if n:
        first = int(np.flatnonzero(mask)[0])
        out.append("{}: {} descriptor(s), first at {}".format(what, n, first))


def _phase2(ph2, nids, ncoef, dims, out, nop=None, lin_acc_bit=False):
    """Checks shared by both Phase-2 forms; nop = the no-op descriptor, if
    the form has one."""
    w = ph2.astype(np.int64)
    kind = w[:, 0] & 3
    if nop is not None:
        isnop = kind == 3
        _bad(isnop & np.any(ph2 != nop, axis=1), "phase 2: malformed no-op", out)
    else:
        _bad(kind == 3, "phase 2: unknown descriptor kind", out)
    dst = w[:, 0] >> 16
    lo1, hi1, lo2, hi2 = w[:, 1] & 0xFFFF, w[:, 1] >> 16, w[:, 2] & 0xFFFF, w[:, 2] >> 16
    hrr = kind == 0
    _bad(hrr & ((dst >= nids) | (lo1 >= nids) | (hi1 >= nids)), "HRR id out of range", out)
    _bad(hrr & (w[:, 2] >= 6), "HRR axis out of range", out)
    lin = kind == 1
    nt = (w[:, 0] >> 2) & 7
    _bad(lin & ((nt < 1) | (nt > 4)), "linear combination with a bad term count", out)
    ops = np.stack([lo1, hi1, lo2, hi2], axis=1)
    coef = np.stack([w[:, 3] & 255, (w[:, 3] >> 8) & 255, (w[:, 3] >> 16) & 255, w[:, 3] >> 24], axis=1)
    used = np.arange(4)[None, :] < nt[:, None]
    _bad(lin & (dst >= nids), "linear combination destination out of range", out)
    _bad(lin & np.any(used & (ops >= nids), axis=1), "linear combination operand out of range", out)
    _bad(lin & np.any(used & (coef >= ncoef), axis=1), "transform coefficient index out of range", out)
    if not lin_acc_bit:
        _bad(lin & (((w[:, 0] >> 5) & 0x7FF) != 0), "linear combination with stray flag bits", out)
    st = kind == 2
    nout = int(np.prod(dims))
    _bad(st & (dst >= nids), "store source out of range", out)
    k = w[:, 1]
    _bad(st & ((k < 0) | (k >= nout)), "store element out of range", out)
    idx = np.stack([w[:, 2] & 255, (w[:, 2] >> 8) & 255, (w[:, 2] >> 16) & 255, w[:, 2] >> 24], axis=1)
    d = np.asarray(dims, dtype=np.int64)
    _bad(st & np.any(idx >= d[None, :], axis=1), "store component index out of range", out)
    flat = ((idx[:, 0] * d[1] + idx[:, 1]) * d[2] + idx[:, 2]) * d[3] + idx[:, 3]
    _bad(st & (flat != k), "store element does not match its component indexes", out)


def verify_coop(cp, L, ncoef):
    """Bounds of a team-cooperative program (gen.coop.CoopProgram) of a class
    of total angular momentum L, against a transform table of ncoef
    entries."""
    out = []
    W = cp.T * cp.ilp
    for name, ph, steps in (("phase 1", cp.ph1, cp.steps1), ("phase 2", cp.ph2, cp.steps2)):
        if ph.ndim != 2 or ph.shape[1] != 4:
            out.append("{}: descriptors are not [n][4]".format(name))
            return out
        if ph.shape[0] != (int(np.sum(steps)) + PREFETCH_STEPS) * W:
            out.append("{}: {} descriptors for {} steps of {} lanes x {}".format(
                name, ph.shape[0], int(np.sum(steps)), cp.T, cp.ilp))
            return out
        if np.any(np.asarray(steps) < (1 if getattr(cp, "lag", 1) == 1 else 0)):
            out.append("{}: empty wave".format(name))
        nop = NOP1 if name == "phase 1" else NOP2
        if np.any(ph[ph.shape[0] - PREFETCH_STEPS * W:] != nop[None, :]):
            out.append("{}: prefetch steps are not no-ops".format(name))
    nslot, nh = cp.nslot, cp.nh
    # ---- Phase 1
    w = cp.ph1.astype(np.int64)
    meta = w[:, 3] >> 16
    nop = (meta & 0x8000) != 0
    _bad(nop & np.any(cp.ph1 != NOP1[None, :], axis=1), "phase 1: malformed no-op", out)
    live = ~nop
    dst = w[:, 0] & 0xFFFF
    h = w[:, 0] >> 16
    _bad(live & (dst != 0xFFFF) & (dst >= nslot), "phase 1: destination slot out of range", out)
    _bad(live & (h > nh), "phase 1: accumulator out of range", out)
    base = live & ((meta & 0x4000) != 0)
    k = (meta >> 4) & 31
    _bad(base & (k > L), "phase 1: Boys order above L", out)
    term = live & ~base
    cgo, k3, side = meta & 15, (meta >> 9) & 15, (meta >> 13) & 1
    _bad(term & ((cgo % 6 >= 3) | (cgo // 6 != side) | (cgo >= 12)), "phase 1: bad side / axis", out)
    _bad(term & ((k > MAX_K) | (k3 > MAX_K)), "phase 1: k or k3 above 8", out)
    s0, s1, s2, s3, s4 = w[:, 1] & 0xFFFF, w[:, 1] >> 16, w[:, 2] & 0xFFFF, w[:, 2] >> 16, w[:, 3] & 0xFFFF
    _bad(term & ((s0 >= nslot) | (s1 >= nslot)), "phase 1: operand slot out of range", out)
    _bad(term & (k > 0) & ((s2 >= nslot) | (s3 >= nslot)), "phase 1: second-term operand out of range", out)
    _bad(term & (k3 > 0) & (s4 >= nslot), "phase 1: cross-term operand out of range", out)
    # largest coefficient-row entry a node reads: 28 + 8 side + k <= 44, 44 + k3 <= 52
    assert 28 + 8 + MAX_K < ROW_ENTRIES and 44 + MAX_K < ROW_ENTRIES
    hs = h[live & (h > 0)]
    _bad(np.bincount(hs, minlength=1)[hs] > 1, "phase 1: accumulator with more than one owner", out)
    # every accumulator has an owner (Phase 2 reads all of H)
    if np.unique(hs).size != nh:
        out.append("phase 1: {} of {} accumulators have no owner".format(nh - np.unique(hs).size, nh))
    # ---- Phase 2
    _phase2(cp.ph2, nh + nslot, ncoef, cp.out_dims, out, nop=NOP2)
    # ---- hazards between and within waves
    lag = getattr(cp, "lag", 1)
    for name, reads, writes in (("phase 1",) + _phase1_access(cp), ("phase 2",) + _phase2_access(cp)):
        prev_r = prev_w = None
        for wv, (r, wr) in enumerate(zip(reads, writes)):
            if np.intersect1d(r, wr).size or np.unique(wr).size != wr.size:
                out.append("{}: wave {} reads a slot it writes, or writes one twice".format(name, wv))
            if lag == 2 and prev_r is not None and (np.intersect1d(r, prev_w).size or
                                                    np.intersect1d(wr, prev_r).size or
                                                    np.intersect1d(wr, prev_w).size):
                out.append("{}: waves {} and {} share a slot under split barriers".format(name, wv - 1, wv))
            prev_r, prev_w = r, wr
    return out


def _waves_of(ph, steps, W):
    i = 0
    for st in np.asarray(steps).tolist():
        yield ph[i:i + int(st) * W].astype(np.int64)
        i += int(st) * W


def _phase1_access(cp):
    """Per wave: value slots read (operands of the terms each node
    evaluates) and written (kept results)."""
    reads, writes = [], []
    for w in _waves_of(cp.ph1, cp.steps1, cp.T * cp.ilp):
        meta = w[:, 3] >> 16
        term = (meta & 0xC000) == 0
        k, k3 = (meta >> 4) & 31, (meta >> 9) & 15
        r = [w[term, 1] & 0xFFFF, w[term, 1] >> 16, w[term & (k > 0), 2] & 0xFFFF, w[term & (k > 0), 2] >> 16,
             w[term & (k3 > 0), 3] & 0xFFFF]
        dst = w[:, 0] & 0xFFFF
        reads.append(np.unique(np.concatenate(r)))
        writes.append(dst[((meta & 0x8000) == 0) & (dst != 0xFFFF)])
    return reads, writes


def _phase2_access(cp):
    """Per wave: operand ids read (accumulators and value slots) and value
    ids written (results of HRR steps and linear combinations)."""
    reads, writes = [], []
    for w in _waves_of(cp.ph2, cp.steps2, cp.T * cp.ilp):
        kind = w[:, 0] & 3
        nt = (w[:, 0] >> 2) & 7
        ops = np.stack([w[:, 1] & 0xFFFF, w[:, 1] >> 16, w[:, 2] & 0xFFFF, w[:, 2] >> 16], axis=1)
        used = np.zeros(ops.shape, dtype=bool)
        used[kind == 0, :2] = True
        used[kind == 1] = np.arange(4)[None, :] < nt[kind == 1, None]
        r = [ops[used], (w[kind == 2, 0] >> 16)]
        reads.append(np.unique(np.concatenate(r)))
        writes.append(w[(kind == 0) | (kind == 1), 0] >> 16)
    return reads, writes


def verify_encoded(enc, ncoef):
    """Bounds of an encoded program (gen.encode.Encoded) for the
    thread-per-quartet executor: one slot space of enc.nslot ids."""
    out = []
    n = enc.nslot
    w = enc.ph1.astype(np.int64)
    if w.size:
        store = ((w[:, 3] >> 30) & 1) != 0
        dst = w[:, 0] & 0xFFFF
        h = w[:, 0] >> 16
        _bad(store & (dst >= n), "phase 1: destination slot out of range", out)
        _bad(h > enc.nh, "phase 1: accumulator out of range", out)
        side = (w[:, 3] >> 16) & 3
        axis = (w[:, 3] >> 18) & 3
        k = (w[:, 3] >> 20) & 31
        k3 = (w[:, 3] >> 25) & 31
        base = side == 2
        _bad(side == 3, "phase 1: bad side", out)
        _bad(base & (k > enc.L), "phase 1: Boys order above L", out)
        term = ~base
        _bad(term & (axis >= 3), "phase 1: axis out of range", out)
        _bad(term & ((k > MAX_K) | (k3 > MAX_K)), "phase 1: k or k3 above 8", out)
        s0, s1, s2, s3, s4 = w[:, 1] & 0xFFFF, w[:, 1] >> 16, w[:, 2] & 0xFFFF, w[:, 2] >> 16, w[:, 3] & 0xFFFF
        _bad(term & ((s0 >= n) | (s1 >= n)), "phase 1: operand slot out of range", out)
        _bad(term & (k > 0) & ((s2 >= n) | (s3 >= n)), "phase 1: second-term operand out of range", out)
        _bad(term & (k3 > 0) & (s4 >= n), "phase 1: cross-term operand out of range", out)
    if enc.ph2.size:
        _phase2(enc.ph2, n, ncoef, enc.out_dims, out, lin_acc_bit=True)
    return out


def check(ls, problems):
    if problems:
        raise ValueError("class {}: program out of bounds: {}".format(ls, "; ".join(problems)))
