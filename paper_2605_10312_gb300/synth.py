"""Seeded synthetic inputs for the contracted-ERI path.

This module holds random numbers and geometry only: molecule layouts, shell
lists, primitive exponents and contraction coefficients, quartet lists.  It
contains none of the integral arithmetic (no normalisation, no Gaussian
products, no recurrences), so both the CPU oracle and the CUDA path may use it.

Units: the workload recipes are stated in Angstrom and converted here to bohr
(1 bohr = 0.529177210903 Angstrom, CODATA 2018); every array handed out is in
bohr.

A ``Basis`` is a flat, C-friendly description:

* ``centers``   float64 [ncenter, 3]   bohr
* ``shell_l``   int32   [nshell]       angular momentum, 0..4
* ``shell_nprim`` int32 [nshell]       contraction depth K
* ``shell_center`` int32 [nshell]      index into ``centers``
* ``shell_prim`` int32  [nshell]       offset of the shell's first primitive
* ``exps``      float64 [nprim_total]  primitive exponents (bohr^-2)
* ``coefs``     float64 [nprim_total]  raw contraction coefficients; the
                                       primitive normalisation is applied by
                                       the integral code, not here.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

ANGSTROM_TO_BOHR = 1.0 / 0.529177210903

L_LETTER = "spdfg"


@dataclass
class Basis:
    centers: np.ndarray
    shell_l: np.ndarray
    shell_nprim: np.ndarray
    shell_center: np.ndarray
    shell_prim: np.ndarray
    exps: np.ndarray
    coefs: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nshell(self) -> int:
        return int(self.shell_l.shape[0])

    def validate(self) -> None:
        assert self.centers.dtype == np.float64 and self.centers.ndim == 2 and self.centers.shape[1] == 3
        for a in (self.shell_l, self.shell_nprim, self.shell_center, self.shell_prim):
            assert a.dtype == np.int32 and a.shape == (self.nshell,)
        assert self.exps.dtype == np.float64 and self.coefs.dtype == np.float64
        assert np.all(self.shell_prim + self.shell_nprim <= self.exps.shape[0])


class _BasisBuilder:
    def __init__(self):
        self.centers: list = []
        self.l: list = []
        self.k: list = []
        self.c: list = []
        self.p: list = []
        self.exps: list = []
        self.coefs: list = []

    def add_center(self, xyz) -> int:
        self.centers.append(np.asarray(xyz, dtype=np.float64))
        return len(self.centers) - 1

    def add_shell(self, l: int, center: int, exps, coefs) -> int:
        exps = np.asarray(exps, dtype=np.float64)
        coefs = np.asarray(coefs, dtype=np.float64)
        assert exps.shape == coefs.shape and exps.ndim == 1 and exps.size >= 1
        self.l.append(l)
        self.k.append(exps.size)
        self.c.append(center)
        self.p.append(sum(len(e) for e in self.exps))
        self.exps.append(exps)
        self.coefs.append(coefs)
        return len(self.l) - 1

    def build(self, **meta) -> Basis:
        b = Basis(
            centers=np.ascontiguousarray(np.array(self.centers, dtype=np.float64).reshape(-1, 3)),
            shell_l=np.array(self.l, dtype=np.int32),
            shell_nprim=np.array(self.k, dtype=np.int32),
            shell_center=np.array(self.c, dtype=np.int32),
            shell_prim=np.array(self.p, dtype=np.int32),
            exps=np.concatenate(self.exps) if self.exps else np.zeros(0),
            coefs=np.concatenate(self.coefs) if self.coefs else np.zeros(0),
            meta=dict(meta),
        )
        b.validate()
        return b


def log_uniform(rng: np.random.Generator, lo: float, hi: float, n: int) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))


def all_unique_quartets(nshell: int) -> np.ndarray:
    """Every shell quartet (ab|cd) with a >= b, c >= d and pair(ab) >= pair(cd):
    one representative per 8-fold permutation orbit."""
    pairs = [(a, b) for a in range(nshell) for b in range(a + 1)]
    out = [(p[0], p[1], q[0], q[1]) for i, p in enumerate(pairs) for q in pairs[: i + 1]]
    return np.array(out, dtype=np.int32).reshape(-1, 4)


# ---------------------------------------------------------------------------
# Workload: tiny plain FP64 set (3 atoms, s s p shells, K = 3)
# ---------------------------------------------------------------------------
def tiny_set(seed: int = 1, natom: int = 3, box_angstrom: float = 3.0, nprim: int = 3):
    """3 atoms uniform in a 3 Angstrom cube; each atom carries two s shells and
    one p shell of 3 primitives, exponents log-uniform in [0.1, 100], raw
    coefficients uniform in [0.1, 1].  Returns (basis, all unique quartets)."""
    rng = np.random.default_rng(seed)
    bb = _BasisBuilder()
    for _ in range(natom):
        c = bb.add_center(rng.uniform(0.0, box_angstrom, size=3) * ANGSTROM_TO_BOHR)
        for l in (0, 0, 1):
            bb.add_shell(l, c, log_uniform(rng, 0.1, 100.0, nprim), rng.uniform(0.1, 1.0, size=nprim))
    basis = bb.build(workload="tiny", seed=seed)
    return basis, all_unique_quartets(basis.nshell)


# ---------------------------------------------------------------------------
# Workload: per-class sweep (independent random quartets of one class)
# ---------------------------------------------------------------------------
def class_sweep(ls, nquartet: int, kset=(1,), seed: int = 2000, box_angstrom: float = 10.0,
                exp_range=(0.05, 500.0), coef_range=(0.1, 1.0)):
    """``nquartet`` independent shell quartets of class ``ls = (la, lb, lc, ld)``.

    Each quartet has four fresh centres uniform in a 10 Angstrom cube and four
    fresh shells; each shell's contraction depth K is drawn uniformly from
    ``kset`` (a single value gives a fixed-K run), exponents log-uniform in
    [0.05, 500], coefficients uniform in [0.1, 1].  Quartet q uses shells
    4q..4q+3 in (a, b, c, d) order."""
    rng = np.random.default_rng(seed)
    ls = tuple(int(x) for x in ls)
    kset = np.asarray(kset, dtype=np.int64)
    n = int(nquartet)
    centers = rng.uniform(0.0, box_angstrom, size=(4 * n, 3)) * ANGSTROM_TO_BOHR
    kk = kset[rng.integers(0, kset.size, size=4 * n)] if kset.size > 1 else np.full(4 * n, kset[0])
    prim = np.zeros(4 * n, dtype=np.int64)
    prim[1:] = np.cumsum(kk)[:-1]
    ntot = int(kk.sum())
    exps = log_uniform(rng, exp_range[0], exp_range[1], ntot)
    coefs = rng.uniform(coef_range[0], coef_range[1], size=ntot)
    basis = Basis(
        centers=np.ascontiguousarray(centers),
        shell_l=np.tile(np.array(ls, dtype=np.int32), n),
        shell_nprim=kk.astype(np.int32),
        shell_center=np.arange(4 * n, dtype=np.int32),
        shell_prim=prim.astype(np.int32),
        exps=exps,
        coefs=coefs,
        meta=dict(workload="class_sweep", ls=ls, kset=tuple(int(k) for k in kset), seed=seed),
    )
    basis.validate()
    quartets = np.arange(4 * n, dtype=np.int32).reshape(n, 4)
    return basis, quartets


def mixed_class_set(classes, nquartet_each: int, kset=(1,), seed: int = 7):
    """Concatenation of several per-class sweeps (one basis, one quartet list),
    quartets interleaved in a seeded random order so that a batch mixes classes."""
    parts = [class_sweep(ls, nquartet_each, kset=kset, seed=seed + 17 * i) for i, ls in enumerate(classes)]
    return concat_sets(parts, shuffle_seed=seed)


def concat_sets(parts, shuffle_seed=None):
    bb_centers, bl, bk, bc, bp, be, bco, qs = [], [], [], [], [], [], [], []
    coff = soff = poff = 0
    for basis, q in parts:
        bb_centers.append(basis.centers)
        bl.append(basis.shell_l)
        bk.append(basis.shell_nprim)
        bc.append(basis.shell_center + coff)
        bp.append(basis.shell_prim + poff)
        be.append(basis.exps)
        bco.append(basis.coefs)
        qs.append(q + soff)
        coff += basis.centers.shape[0]
        soff += basis.nshell
        poff += basis.exps.shape[0]
    basis = Basis(
        centers=np.ascontiguousarray(np.concatenate(bb_centers)),
        shell_l=np.concatenate(bl).astype(np.int32),
        shell_nprim=np.concatenate(bk).astype(np.int32),
        shell_center=np.concatenate(bc).astype(np.int32),
        shell_prim=np.concatenate(bp).astype(np.int32),
        exps=np.concatenate(be),
        coefs=np.concatenate(bco),
        meta=dict(workload="concat"),
    )
    quartets = np.ascontiguousarray(np.concatenate(qs).astype(np.int32))
    if shuffle_seed is not None:
        perm = np.random.default_rng(shuffle_seed).permutation(quartets.shape[0])
        quartets = np.ascontiguousarray(quartets[perm])
    basis.validate()
    return basis, quartets


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix from a uniform unit quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def with_centers(basis: Basis, centers: np.ndarray) -> Basis:
    b = Basis(np.ascontiguousarray(centers, dtype=np.float64), basis.shell_l, basis.shell_nprim,
              basis.shell_center, basis.shell_prim, basis.exps, basis.coefs, dict(basis.meta))
    b.validate()
    return b


# ---------------------------------------------------------------------------
# Workload: water clusters (batched mixed-class and serving workloads)
# ---------------------------------------------------------------------------
# shell layouts per element: (l, K) in order; K runs from 6 for the first s
# shell down to 1 for the polarisation shells
WATER_LAYOUTS = {
    "dz": {"O": [(0, 6), (0, 3), (0, 1), (1, 3), (1, 1), (2, 1)],
           "H": [(0, 3), (0, 1), (1, 1)]},
    "tz": {"O": [(0, 6), (0, 3), (0, 1), (0, 1), (1, 3), (1, 1), (1, 1), (2, 1), (2, 1), (3, 1)],
           "H": [(0, 3), (0, 1), (0, 1), (1, 1), (1, 1), (2, 1)]},
}


def water_positions(nwater: int, rng: np.random.Generator, density=0.02, min_oo=2.8, roh=0.96, angle=104.5):
    """Random sequential insertion of rigid waters (O-H 0.96 A, H-O-H 104.5
    deg, uniform random orientation) with O-O >= 2.8 A in a cube sized for
    `density` molecules per cubic Angstrom.  Returns [3 * nwater, 3] Angstrom,
    ordered O, H, H per molecule."""
    side = (nwater / density) ** (1.0 / 3.0)
    oxy = []
    tries = 0
    while len(oxy) < nwater:
        tries += 1
        if tries > 1000 * nwater:
            raise RuntimeError("could not place the waters")
        p = rng.uniform(0.0, side, size=3)
        if all(np.linalg.norm(p - o) >= min_oo for o in oxy):
            oxy.append(p)
    half = np.deg2rad(angle) / 2.0
    h1 = roh * np.array([np.sin(half), 0.0, np.cos(half)])
    h2 = roh * np.array([-np.sin(half), 0.0, np.cos(half)])
    out = []
    for o in oxy:
        R = random_rotation(rng)
        out.extend([o, o + R @ h1, o + R @ h2])
    return np.array(out)


def element_basis(rng: np.random.Generator, layout):
    """One synthetic basis per element: exponents log-uniform in [0.05, 500]
    sorted tight to diffuse within each shell, coefficients uniform in
    [0.1, 1]."""
    out = {}
    for el in ("O", "H"):
        shells = []
        for l, k in layout[el]:
            exps = np.sort(log_uniform(rng, 0.05, 500.0, k))[::-1]
            shells.append((l, exps, rng.uniform(0.1, 1.0, size=k)))
        out[el] = shells
    return out


def water_cluster(nwater: int, seed: int = 3, layout: str = "dz"):
    """Cluster of `nwater` waters with the per-element shell layout
    (`dz`: O 3s 2p 1d, H 2s 1p; `tz`: O 4s 3p 2d 1f, H 3s 2p 1d).  Returns a
    Basis (atoms O, H, H per molecule) with meta['atoms']."""
    rng = np.random.default_rng(seed)
    pos = water_positions(nwater, rng) * ANGSTROM_TO_BOHR
    eb = element_basis(rng, WATER_LAYOUTS[layout])
    bb = _BasisBuilder()
    for i, p in enumerate(pos):
        el = "O" if i % 3 == 0 else "H"
        c = bb.add_center(p)
        for l, exps, coefs in eb[el]:
            bb.add_shell(l, c, exps, coefs)
    return bb.build(workload="water_cluster", nwater=nwater, seed=seed, layout=layout, atoms=3 * nwater)


def shell_pairs(nshell: int) -> np.ndarray:
    """Unique shell pairs (a >= b), [npair, 2]."""
    a, b = np.tril_indices(nshell)
    return np.stack([a, b], axis=1).astype(np.int32)


def survives(q_p, q_r, p, r, threshold):
    """The screening rule, elementwise: for pairs p, r with factors q_p, q_r,
    lo is the one with the smaller factor (the larger index among equal
    factors) and hi the other; the quartet survives iff
    q_hi >= threshold / q_lo (q_lo = 0: iff threshold <= 0).  Phrased with
    the division so that the sorted-prefix enumeration below, the count and
    a device kernel all pick the same set."""
    q_p, q_r = np.asarray(q_p, dtype=np.float64), np.asarray(q_r, dtype=np.float64)
    p_lo = (q_p < q_r) | ((q_p == q_r) & (np.asarray(p) > np.asarray(r)))
    lo, hi = np.where(p_lo, q_p, q_r), np.where(p_lo, q_r, q_p)
    with np.errstate(divide="ignore"):
        return np.where(lo > 0, hi >= threshold / np.where(lo > 0, lo, 1.0), threshold <= 0)


def screened_quartets(pair_bound: np.ndarray, pairs: np.ndarray, threshold: float) -> np.ndarray:
    """Unique quartets (unordered pairs of pairs, a pair with itself
    included) that pass the screening rule (survives) on the per-pair
    Schwarz bounds; [n, 4] int32, the pair of the smaller bound first.  Pure
    bookkeeping on bounds computed elsewhere."""
    order = np.argsort(-pair_bound, kind="stable")
    qb = pair_bound[order]
    out = []
    for i in range(order.size):
        # nothing from here on has a partner (bounds only fall)
        if (qb[i] > 0 and qb[0] < threshold / qb[i]) or (qb[i] <= 0 and threshold > 0):
            break
        # partners j <= i in the sorted order with qb[i] qb[j] >= threshold:
        # a prefix, since qb is sorted descending
        if qb[i] > 0:
            n = int(np.searchsorted(-qb[: i + 1], -threshold / qb[i], side="right"))
        else:
            n = i + 1 if threshold <= 0 else 0
        if n == 0:
            continue
        P = pairs[order[i]]
        Q = pairs[order[:n]]
        out.append(np.concatenate([np.broadcast_to(P, (n, 2)), Q], axis=1))
    if not out:
        return np.zeros((0, 4), dtype=np.int32)
    return np.ascontiguousarray(np.concatenate(out).astype(np.int32))


def count_screened(pair_bound: np.ndarray, threshold: float) -> int:
    """Number of unique quartets (pair P >= pair Q) with Q_P Q_Q >= threshold."""
    qs = np.sort(np.asarray(pair_bound, dtype=np.float64))[::-1]
    idx = np.arange(qs.size)
    with np.errstate(divide="ignore"):
        lim = np.where(qs > 0, threshold / np.where(qs > 0, qs, 1.0), np.inf if threshold > 0 else -np.inf)
    # partners k <= i with qs[k] >= lim[i]: a prefix of the descending order
    nk = np.searchsorted(-qs, -lim, side="right")
    return int(np.minimum(nk, idx + 1).sum())


def sample_screened_quartets(pair_bound: np.ndarray, pairs: np.ndarray, threshold: float, n: int,
                             seed: int = 0) -> np.ndarray:
    """A uniform random sample (without replacement, seeded) of n unique
    quartets (pair P >= pair Q) whose Schwarz bound Q_P Q_Q >= threshold, for
    screened lists too large to enumerate (all survivors, shuffled, when
    there are at most n).  [m, 4] int32 in random order."""
    rng = np.random.default_rng(seed)
    npair = pair_bound.shape[0]
    ntri = npair * (npair + 1) // 2
    total = count_screened(pair_bound, threshold)
    if n >= total:
        full = screened_quartets(pair_bound, pairs, threshold)
        return np.ascontiguousarray(full[rng.permutation(full.shape[0])])
    frac = total / max(1, ntri)
    got = np.zeros(0, dtype=np.int64)
    while got.size < n:
        m = int(min(max(1.3 * (n - got.size) / max(frac, 1e-12), 1 << 16), 1 << 26))
        t = rng.integers(0, ntri, size=m, dtype=np.int64)
        i = ((np.sqrt(8.0 * t + 1.0) - 1.0) // 2).astype(np.int64)  # triangle index -> (i, j), i >= j
        i -= (i * (i + 1) // 2 > t)
        i += ((i + 1) * (i + 2) // 2 <= t)
        j = t - i * (i + 1) // 2
        t = t[survives(pair_bound[i], pair_bound[j], i, j, threshold)]
        got = np.unique(np.concatenate([got, t]))
    t = rng.permutation(got)[:n]
    i = ((np.sqrt(8.0 * t + 1.0) - 1.0) // 2).astype(np.int64)
    i -= (i * (i + 1) // 2 > t)
    i += ((i + 1) * (i + 2) // 2 <= t)
    j = t - i * (i + 1) // 2
    return np.ascontiguousarray(np.concatenate([pairs[i], pairs[j]], axis=1).astype(np.int32))
