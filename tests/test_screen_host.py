"""Host-side Schwarz screening bookkeeping (no GPU): the surviving quartet
list equals brute force over all unique pair pairs, each exactly once."""
import numpy as np
import pytest

from paper_2605_10312_gb300 import synth


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("thr", [0.0, 1e-12, 1e-6, 1e-2, 10.0])
def test_screened_quartets_brute_force(seed, thr):
    rng = np.random.default_rng(seed)
    nshell = 17
    pairs = synth.shell_pairs(nshell)
    q = 10.0 ** rng.uniform(-9, 0.5, pairs.shape[0])
    q[rng.integers(0, q.size, 5)] = 0.0
    q[3] = q[7]  # ties
    got = synth.screened_quartets(q, pairs, thr)
    want = set()
    for i in range(q.size):
        for j in range(i + 1):
            if q[i] * q[j] >= thr:
                want.add(frozenset([i, j]) if i != j else frozenset([i]))
    index = {tuple(p): k for k, p in enumerate(pairs.tolist())}
    seen = []
    for row in got.tolist():
        a, b = index[tuple(row[:2])], index[tuple(row[2:])]
        assert q[a] * q[b] >= thr
        seen.append(frozenset([a, b]) if a != b else frozenset([a]))
    assert len(seen) == len(set(seen))
    assert set(seen) == want


def test_shell_pairs_unique():
    p = synth.shell_pairs(9)
    assert p.shape == (45, 2)
    assert (p[:, 0] >= p[:, 1]).all()
    assert len({tuple(x) for x in p.tolist()}) == 45


def test_water_cluster_shapes():
    b = synth.water_cluster(20, seed=3, layout="dz")
    assert b.nshell == 240
    assert synth.shell_pairs(b.nshell).shape[0] == 28920
    t = synth.water_cluster(2, seed=3, layout="tz")
    assert t.shell_l.max() == 3


def test_sample_screened_quartets():
    rng = np.random.default_rng(3)
    pairs = synth.shell_pairs(30)
    q = 10.0 ** rng.uniform(-8, 0, pairs.shape[0])
    thr = 1e-6
    full = synth.screened_quartets(q, pairs, thr)
    index = {tuple(p): k for k, p in enumerate(pairs.tolist())}

    def key(row):
        a, b = index[tuple(row[:2])], index[tuple(row[2:])]
        return (max(a, b), min(a, b))
    want = {key(r) for r in full.tolist()}
    s = synth.sample_screened_quartets(q, pairs, thr, 500, seed=1)
    got = [key(r) for r in s.tolist()]
    assert len(got) == 500 and len(set(got)) == 500
    assert set(got) <= want
    # asking for more than survive returns every survivor once
    s_all = synth.sample_screened_quartets(q, pairs, thr, len(want) + 10, seed=2)
    assert {key(r) for r in s_all.tolist()} == want and s_all.shape[0] == len(want)
    # same seed, same sample
    assert np.array_equal(s, synth.sample_screened_quartets(q, pairs, thr, 500, seed=1))


@pytest.mark.parametrize("thr", [0.0, 1e-9, 1e-4, 1.0])
def test_count_screened(thr):
    rng = np.random.default_rng(5)
    pairs = synth.shell_pairs(20)
    q = 10.0 ** rng.uniform(-8, 0.3, pairs.shape[0])
    q[:4] = 0.0
    assert synth.count_screened(q, thr) == synth.screened_quartets(q, pairs, thr).shape[0]


def test_water_cluster_geometry_and_basis():
    """The recipe of the water-cluster workloads: rigid waters (O-H 0.96 A,
    H-O-H 104.5 deg), O-O >= 2.8 A, one basis per element shared by all its
    atoms, exponents in [0.05, 500] sorted tight to diffuse within a shell,
    coefficients in [0.1, 1]."""
    b = synth.water_cluster(20, seed=3, layout="dz")
    xyz = b.centers / synth.ANGSTROM_TO_BOHR
    assert xyz.shape == (60, 3)
    O, H1, H2 = xyz[0::3], xyz[1::3], xyz[2::3]
    assert np.allclose(np.linalg.norm(H1 - O, axis=1), 0.96, atol=1e-12)
    assert np.allclose(np.linalg.norm(H2 - O, axis=1), 0.96, atol=1e-12)
    cosang = np.sum((H1 - O) * (H2 - O), axis=1) / 0.96 ** 2
    assert np.allclose(np.degrees(np.arccos(cosang)), 104.5, atol=1e-9)
    d = np.linalg.norm(O[:, None] - O[None], axis=2) + np.eye(20) * 1e9
    assert d.min() >= 2.8
    # per atom: O 3s 2p 1d (K = 6, 3, 1, 3, 1, 1), H 2s 1p (K = 3, 1, 1)
    per_atom = {0: [(0, 6), (0, 3), (0, 1), (1, 3), (1, 1), (2, 1)], 1: [(0, 3), (0, 1), (1, 1)]}
    shells = {}
    for s in range(b.nshell):
        shells.setdefault(int(b.shell_center[s]), []).append(s)
    for atom, ss in shells.items():
        want = per_atom[0 if atom % 3 == 0 else 1]
        assert [(int(b.shell_l[s]), int(b.shell_nprim[s])) for s in ss] == want
        ref = shells[0 if atom % 3 == 0 else 1]   # the first atom of the same element
        for s, r in zip(ss, ref):
            e = b.exps[b.shell_prim[s]:b.shell_prim[s] + b.shell_nprim[s]]
            assert np.array_equal(e, b.exps[b.shell_prim[r]:b.shell_prim[r] + b.shell_nprim[r]])
            assert np.all(np.diff(e) < 0) and e.min() >= 0.05 and e.max() <= 500.0
    assert b.coefs.min() >= 0.1 and b.coefs.max() <= 1.0


def test_tiny_set_and_class_sweep_recipes():
    """The tiny set: 3 atoms in a 3 A cube, each with s, s, p shells of 3
    primitives (exponents in [0.1, 100], coefficients in [0.1, 1]), and all
    45 * 46 / 2 = 1035 unique quartets.  The per-class sweep: independent
    quartets of one class, four fresh centres each in a 10 A cube, K per
    shell drawn from the given set, exponents in [0.05, 500]."""
    b, q = synth.tiny_set(seed=1)
    assert b.nshell == 9 and q.shape == (1035, 4)
    assert list(b.shell_l) == [0, 0, 1] * 3 and set(b.shell_nprim.tolist()) == {3}
    xyz = b.centers / synth.ANGSTROM_TO_BOHR
    assert xyz.shape == (3, 3) and xyz.min() >= 0.0 and xyz.max() <= 3.0
    assert b.exps.min() >= 0.1 and b.exps.max() <= 100.0 and b.coefs.min() >= 0.1 and b.coefs.max() <= 1.0
    # unique under the 8-fold permutational symmetry
    canon = {tuple(sorted([tuple(sorted(x[:2])), tuple(sorted(x[2:]))])) for x in q.tolist()}
    assert len(canon) == 1035
    b, q = synth.class_sweep((2, 1, 3, 0), 500, kset=(1, 3, 6), seed=9)
    assert q.shape == (500, 4) and np.array_equal(q.ravel(), np.arange(2000))
    assert list(b.shell_l[:4]) == [2, 1, 3, 0]
    assert set(b.shell_nprim.tolist()) == {1, 3, 6} and np.array_equal(b.shell_center, np.arange(2000))
    xyz = b.centers / synth.ANGSTROM_TO_BOHR
    assert xyz.min() >= 0.0 and xyz.max() <= 10.0
    assert b.exps.min() >= 0.05 and b.exps.max() <= 500.0


def test_screening_rule_by_brute_force():
    """The sorted-prefix enumeration and the count pick exactly the
    unordered pairs of pairs {p, r} (p >= r) that pass the elementwise rule,
    on bounds with ties, zeros and values at the threshold's edge."""
    rng = np.random.default_rng(11)
    for thr in (1e-10, 0.0, 1.0, 3.0e-3):
        q = np.concatenate([10.0 ** rng.uniform(-8, 0, 40), np.zeros(3), np.full(4, 0.05), [np.sqrt(thr) if thr else 0]])
        rng.shuffle(q)
        npair = q.size
        pairs = np.stack([np.arange(npair), np.arange(npair)], axis=1).astype(np.int32)   # pair id in both columns
        p, r = np.tril_indices(npair)
        keep = synth.survives(q[p], q[r], p, r, thr)
        want = {(int(a), int(b)) for a, b in zip(p[keep], r[keep])}
        got = synth.screened_quartets(q, pairs, thr)
        got_set = {(max(int(x[0]), int(x[2])), min(int(x[0]), int(x[2]))) for x in got}
        assert got.shape[0] == len(got_set) == len(want) and got_set == want
        assert synth.count_screened(q, thr) == len(want)
