"""Phase 2 of the HGP scheme: the horizontal recurrence (FusionRCG Eq. 3 on
the bra, its mirror on the ket) with the Cartesian-to-spherical transform
(Eq. 8).

Input is the contracted accumulator bank H[e][f] (e of degree la..la+lb on
centre A, f of degree lc..lc+ld on centre C).  Three modes:

  "stepwise"    the fused operator of Eq. 16:
                (T_c x T_d) R_cd (T_a x T_b) R_ab H, one index at a time
                (mask 0000 -> 1000 -> 1100 -> 1110 -> 1111, Fig. 4);
  "materialize" Eq. 17: both HRR sweeps on Cartesian tensors, then the four
                one-index transforms;
  "cart"        both HRR sweeps, Cartesian output (the "No spherical"
                ablation).

The result is a list of straight-line operations on value ids:
  ("hrr", dst, hi, ("AB"|"CD", axis), lo)    dst = hi + X_axis * lo
  ("lin", dst, [(coef, src), ...])            dst = sum coef * src
Value ids 0..NH-1 are the accumulators H (row-major [ie][jf]).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import cart, sph

MODES = ("stepwise", "materialize", "cart")


@dataclass
class Phase2:
    ops: list = field(default_factory=list)
    nvals: int = 0
    outputs: list = field(default_factory=list)   # value id per output element
    out_dims: tuple = ()
    alias_count: int = 0

    def new(self) -> int:
        self.nvals += 1
        return self.nvals - 1


def _hrr_axis(b, rule):
    if rule == "first":
        return next(i for i in range(3) if b[i] > 0)
    if rule == "last":
        return next(i for i in (2, 1, 0) if b[i] > 0)
    if rule == "max":
        m = max(b)
        return next(i for i in (2, 1, 0) if b[i] == m)
    raise ValueError(rule)


def _hrr_pair(P, l1, l2, src, sym, rule):
    """One HRR sweep for a fixed other index: src maps tuple e (degree
    l1..l1+l2) to a value id; returns {(a, b): value id} for |a| = l1, |b| = l2."""
    memo = {}
    z3 = (0, 0, 0)

    def val(e, b):
        if b == z3:
            return src[e]
        key = (e, b)
        if key in memo:
            return memo[key]
        i = _hrr_axis(b, rule)
        hi = val(cart.add(e, i), cart.sub(b, i))
        lo = val(e, cart.sub(b, i))
        d = P.new()
        P.ops.append(("hrr", d, hi, (sym, i), lo))
        memo[key] = d
        return d

    return {(a, b): val(a, b) for a in cart.tuples(l1) for b in cart.tuples(l2)}


def _transform(P, l, get, n_other):
    """One-index transform T^(l) applied to index values get(alpha, o) for
    o in range(n_other); returns out[mu][o] value ids.  Rows of T with a
    single unit coefficient become aliases (no operation)."""
    T = sph.matrix(l)
    out = [[None] * n_other for _ in range(T.shape[0])]
    for mu in range(T.shape[0]):
        nz = [(float(T[mu, a]), a) for a in range(T.shape[1]) if T[mu, a] != 0.0]
        for o in range(n_other):
            if len(nz) == 1 and nz[0][0] == 1.0:
                out[mu][o] = get(nz[0][1], o)
                P.alias_count += 1
            else:
                d = P.new()
                P.ops.append(("lin", d, [(c, get(a, o)) for c, a in nz]))
                out[mu][o] = d
    return out


def build(la, lb, lc, ld, mode="stepwise", rule="first") -> Phase2:
    if mode not in MODES:
        raise ValueError(mode)
    E = cart.range_tuples(la, la + lb)
    F = cart.range_tuples(lc, lc + ld)
    nf = len(F)
    P = Phase2(nvals=len(E) * nf)
    ta, tb, tc, td = (cart.tuples(x) for x in (la, lb, lc, ld))
    ia = {t: k for k, t in enumerate(E)}

    sa, sb, scn, sdn = 2 * la + 1, 2 * lb + 1, 2 * lc + 1, 2 * ld + 1
    na, nb, nc, nd = len(ta), len(tb), len(tc), len(td)
    if mode == "stepwise":
        # column by column: bra HRR for ket tuple f, then T_a, then T_b
        # (mask 0000 -> 1000 -> 1100), so that only the spherical bra half
        # of finished columns stays live
        bra_vals = {(mu, nu): {} for mu in range(sa) for nu in range(sb)}
        for jf in range(nf):
            src = {e: ia[e] * nf + jf for e in E}
            res = _hrr_pair(P, la, lb, src, "AB", rule)
            g1 = {(cart.index(a), cart.index(b)): v for (a, b), v in res.items()}
            Ga = _transform(P, la, lambda al, o: g1[(al, o)], nb)          # Ga[mu][beta]
            Gb = _transform(P, lb, lambda be, o: Ga[o][be], sa)            # Gb[nu][mu]
            for mu in range(sa):
                for nu in range(sb):
                    bra_vals[(mu, nu)][F[jf]] = Gb[nu][mu]
        # bra pair by bra pair: ket HRR, then T_c, then T_d (1110 -> 1111)
        out = []
        for mu in range(sa):
            for nu in range(sb):
                res = _hrr_pair(P, lc, ld, bra_vals[(mu, nu)], "CD", rule)
                g3 = {(cart.index(c), cart.index(d)): v for (c, d), v in res.items()}
                Gc = _transform(P, lc, lambda g, o: g3[(g, o)], nd)        # Gc[lam][delta]
                Gd = _transform(P, ld, lambda d, o: Gc[o][d], scn)         # Gd[sig][lam]
                for lam in range(scn):
                    for sig in range(sdn):
                        out.append(Gd[sig][lam])
        P.outputs = out
        P.out_dims = (sa, sb, scn, sdn)
        return P

    # bra HRR for every ket tuple f
    G1 = {}  # (ca, cb, jf) -> id
    for jf in range(nf):
        src = {e: ia[e] * nf + jf for e in E}
        res = _hrr_pair(P, la, lb, src, "AB", rule)
        for (a, b), v in res.items():
            G1[(cart.index(a), cart.index(b), jf)] = v
    bra_vals = {}
    for ca in range(na):
        for cb in range(nb):
            bra_vals[(ca, cb)] = {F[jf]: G1[(ca, cb, jf)] for jf in range(nf)}
    nbra = (na, nb)

    # ket HRR for every bra pair
    G3 = {}  # (bra pair, cc, cd) -> id
    for bp, src in bra_vals.items():
        res = _hrr_pair(P, lc, ld, src, "CD", rule)
        for (c, d), v in res.items():
            G3[(bp, cart.index(c), cart.index(d))] = v
    bras = [(i, j) for i in range(nbra[0]) for j in range(nbra[1])]

    if mode == "cart":
        P.outputs = [G3[(bp, c, d)] for bp in bras for c in range(nc) for d in range(nd)]
        P.out_dims = (len(ta), len(tb), nc, nd)
    else:  # materialize: four one-index transforms of the full Cartesian tensor
        dims = [len(ta), len(tb), nc, nd]
        cur = {}
        for (i, j) in bras:
            for c in range(nc):
                for d in range(nd):
                    cur[(i, j, c, d)] = G3[((i, j), c, d)]
        for w, l in enumerate((la, lb, lc, ld)):
            others = [k for k in range(4) if k != w]
            idx_other = list(np.ndindex(*[dims[k] for k in others]))

            def get(al, o, w=w, others=others, idx_other=idx_other):
                key = [0, 0, 0, 0]
                key[w] = al
                for k, v in zip(others, idx_other[o]):
                    key[k] = v
                return cur[tuple(key)]

            res = _transform(P, l, get, len(idx_other))
            new = {}
            for mu in range(2 * l + 1):
                for o, io in enumerate(idx_other):
                    key = [0, 0, 0, 0]
                    key[w] = mu
                    for k, v in zip(others, io):
                        key[k] = v
                    new[tuple(key)] = res[mu][o]
            dims[w] = 2 * l + 1
            cur = new
        P.outputs = [cur[k] for k in np.ndindex(*dims)]
        P.out_dims = tuple(dims)
    return P


def op_counts(P: Phase2):
    """(instructions, flops): an HRR step is one FMA (2 flops); a transform
    row of n terms is one multiply and n-1 FMAs."""
    ins = fl = 0
    for op in P.ops:
        if op[0] == "hrr":
            ins += 1
            fl += 2
        else:
            n = len(op[2])
            ins += n
            fl += 2 * n - 1
    return ins, fl


def best(la, lb, lc, ld, mode="stepwise"):
    """The HRR axis rule with the fewest operations for this class."""
    cands = [build(la, lb, lc, ld, mode, r) for r in ("first", "last", "max")]
    return min(cands, key=lambda P: op_counts(P)[0])
