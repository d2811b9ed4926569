"""A class program: everything the emitter needs for one angular-momentum
class (la, lb, lc, ld) in its evaluation orientation -- recurrences build on
centres A and C, HRR moves angular momentum to B and D.

Operation counts follow one convention throughout (FMA = 2 flops, a single
add or multiply = 1); the contraction add is folded into the first
multiply of every target's Phase-1 expression, so it costs no instruction.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from functools import lru_cache

from . import cart, hrr, vrr

# per-primitive-quartet setup, counted from the device code in
# eri_common.cuh (pair quantities come precomputed per primitive pair):
# 1/(zeta+eta), P-Q, rho, W-P, W-Q, T, sqrt for the prefactor, prefactor.
SETUP_FLOPS = 24
# Boys: 8-term Taylor (16) + exp + downward recursion (2 per order) or
# asymptotic start + upward recursion (2 per order); exp/sqrt/rcp = 1.
BOYS_BASE_FLOPS = 18


@dataclass
class Options:
    axis_rule: str = "prose"
    schedule: str = "dsa"
    sph_mode: str = "stepwise"

    def key(self):
        return (self.axis_rule, self.schedule, self.sph_mode)


@dataclass
class ClassProgram:
    ls: tuple
    opts: Options
    g: vrr.VrrGraph
    order: list
    peak: int
    slot: list
    nslot: int
    p2: hrr.Phase2
    coef_syms: set = field(default_factory=set)

    @property
    def L(self):
        return sum(self.ls)

    @property
    def nh(self):
        E, F = vrr.h_layout(*self.ls)
        return len(E) * len(F)

    @property
    def nout(self):
        n = 1
        for d in self.p2.out_dims:
            n *= d
        return n

    def vrr_counts(self):
        """(instructions, flops) of Phase 1 for one primitive quartet,
        including the base values pref * F_m and the folded contraction."""
        ins = fl = 0
        for v in self.order:
            nt = len(self.g.terms[v])
            if nt == 0:
                ins += 1
                fl += 1
                continue
            ins += nt
            fl += 2 * nt - 1 + (1 if v in self.g.target else 0)
        return ins, fl

    def counts(self, K4=1):
        """Algorithmic flops for one shell quartet with K4 primitive quartets."""
        vi, vf = self.vrr_counts()
        pi, pf = hrr.op_counts(self.p2)
        coef = len(self.coef_syms)
        per_prim = SETUP_FLOPS + BOYS_BASE_FLOPS + 2 * self.L + coef + vf
        return dict(vrr_nodes=len(self.g), vrr_instr=vi, vrr_flops=vf, p2_instr=pi, p2_flops=pf,
                    per_prim_flops=per_prim, flops=K4 * per_prim + pf, peak_live=self.peak, nslot=self.nslot,
                    nh=self.nh, nout=self.nout)


@lru_cache(maxsize=None)
def make(la, lb, lc, ld, axis_rule="prose", schedule="dsa", sph_mode="stepwise") -> ClassProgram:
    opts = Options(axis_rule, schedule, sph_mode)
    g = vrr.build(la, lb, lc, ld, axis_rule)
    order = vrr.schedule(g, schedule)
    peak = vrr.peak_live(g, order)
    slot, nslot = vrr.allocate_slots(g, order)
    p2 = hrr.best(la, lb, lc, ld, sph_mode)
    syms = set()
    for ts in g.terms:
        for c, _ in ts:
            syms.add(c)
    return ClassProgram((la, lb, lc, ld), opts, g, order, peak, list(map(int, slot)), int(nslot), p2, syms)


def all_classes(lmax=4):
    """Every class in evaluation orientation: ordered bra pair (la, lb) and
    ordered ket pair (lc, ld), with bra-ket exchange symmetry removed
    (pair index of the bra >= that of the ket): 25 * 26 / 2 = 325 for lmax 4."""
    pairs = [(a, b) for a in range(lmax + 1) for b in range(lmax + 1)]
    out = []
    for i, p in enumerate(pairs):
        for q in pairs[: i + 1]:
            out.append(p + q)
    return out


def pair_rank(la, lb, lmax=4):
    return la * (lmax + 1) + lb
