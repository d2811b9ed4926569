"""Parity of the CUDA path with the CPU oracle, element by element, within
|d| <= max(1e-12, 1e-10 |ref|) (the FP64 tolerance of the ERI path)."""
import itertools

import numpy as np
import pytest

from paper_2605_10312_gb300 import synth
from ref import adjudicated, report, within

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eri():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_10312_gb300 import eri as m
    m.library()
    return m


def _run(eri, basis, q, **opts):
    got, off = eri.eri(basis, q, **opts)
    return got.cpu().numpy(), off


def test_tiny_set_all_quartets(eri):
    """3 atoms x (s, s, p), K = 3: every unique quartet (1035)."""
    basis, q = synth.tiny_set(seed=1)
    assert q.shape[0] == 1035
    got, off = _run(eri, basis, q)
    ref, roff = adjudicated(got, basis, q)
    assert np.array_equal(off, roff)
    assert within(got, ref).all(), report(got, ref)


ALL_LS = list(itertools.product(range(5), repeat=4))


@pytest.mark.parametrize("chunk", range(5))
def test_every_class_compact(eri, chunk):
    """All 625 ordered (la lb | lc ld) combinations (every one of the 325
    classes in both pair orientations), K in {1, 2}, compact geometry."""
    parts = [synth.class_sweep(ls, 2, kset=(1, 2), seed=10000 + i, box_angstrom=3.0, exp_range=(0.1, 60.0))
             for i, ls in enumerate(ALL_LS) if i % 5 == chunk]
    basis, q = synth.concat_sets(parts, shuffle_seed=chunk)
    got, _ = _run(eri, basis, q)
    ref, _ = adjudicated(got, basis, q)
    assert within(got, ref).all(), report(got, ref)


@pytest.mark.parametrize("ls", [(1, 1, 1, 1), (2, 2, 2, 2), (3, 3, 3, 3), (4, 4, 4, 4)])
def test_sweep_classes(eri, ls):
    """The per-class sweep geometry (10 Angstrom box, exponents in
    [0.05, 500]), contraction depth per shell drawn from {1, 3, 6}."""
    n = {1: 600, 2: 200, 3: 24, 4: 6}[ls[0]]
    kset = (1, 3, 6) if ls[0] <= 2 else (1, 3)
    basis, q = synth.class_sweep(ls, n, kset=kset, seed=2000 + ls[0])
    got, _ = _run(eri, basis, q)
    ref, _ = adjudicated(got, basis, q)
    assert within(got, ref).all(), report(got, ref)
    # the sweep geometry makes most integrals tiny: also hold the relative
    # error on the larger half of each block to 1e-10
    big = np.abs(ref) > 1e-3 * np.abs(ref).max()
    assert (np.abs(got - ref)[big] <= 1e-10 * np.abs(ref)[big] + 1e-14).all()


def test_deep_contraction(eri):
    """K = 6 on every shell (1296 primitive quartets per shell quartet) and
    K up to 12 on mixed shells."""
    basis, q = synth.class_sweep((2, 1, 2, 0), 8, kset=(6,), seed=77, box_angstrom=3.0)
    got, _ = _run(eri, basis, q)
    ref, _ = adjudicated(got, basis, q)
    assert within(got, ref).all(), report(got, ref)
    basis, q = synth.class_sweep((1, 1, 0, 1), 8, kset=(1, 7, 12), seed=78, box_angstrom=3.0)
    got, _ = _run(eri, basis, q)
    ref, _ = adjudicated(got, basis, q)
    assert within(got, ref).all(), report(got, ref)


def test_ragged_batch_sizes(eri):
    """Quartet counts that leave partial blocks and partial waves."""
    for n in (1, 31, 129, 1000, 4097):
        basis, q = synth.class_sweep((1, 0, 1, 0), n, kset=(1, 3), seed=300 + n, box_angstrom=3.0)
        got, _ = _run(eri, basis, q)
        ref, _ = adjudicated(got, basis, q)
        assert within(got, ref).all(), (n, report(got, ref))


def test_permutations_agree(eri):
    """All eight orderings of the same quartets, transposed back."""
    basis, q = synth.class_sweep((3, 1, 2, 0), 16, kset=(1, 3), seed=5, box_angstrom=3.0)
    perms = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2), (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0),
             (3, 2, 1, 0)]
    base, off = _run(eri, basis, q)
    for p in perms[1:]:
        got, offp = _run(eri, basis, q[:, list(p)])
        for i in range(q.shape[0]):
            dims = [[1, 3, 5, 7, 9][basis.shell_l[s]] for s in q[i][list(p)]]
            b = np.transpose(got[offp[i]:offp[i + 1]].reshape(dims), np.argsort(p)).ravel()
            r = base[off[i]:off[i + 1]]
            assert within(b, r, atol=1e-14, rtol=1e-12).all()


@pytest.mark.parametrize("votes", ["off", "on"])
@pytest.mark.parametrize("ls", [(1, 1, 1, 1), (2, 2, 2, 1), (2, 2, 2, 2), (3, 3, 2, 2), (3, 3, 3, 3), (4, 4, 4, 3),
                                (4, 4, 4, 4)])
def test_cooperative_program_forms(eri, ls, votes):
    """Both forms of the team-cooperative programs -- optional FP64 terms
    predicated per lane, or skipped by a warp none of whose lanes needs
    them -- against the oracle, on deep, shallow and single-primitive
    contractions (K per shell from {1, 2, 6}); (pp|pp) through the
    cooperative tier instead of its compiled kernel."""
    n = {1: 60, 2: 24, 3: 6, 4: 3}[ls[0]]
    basis, q = synth.class_sweep(ls, n, kset=(1, 2, 6) if ls[0] < 4 else (1, 2), seed=90 + sum(ls),
                                 box_angstrom=3.0, exp_range=(0.1, 60.0))
    got, _ = _run(eri, basis, q, votes=votes, tier="coop")
    ref, _ = adjudicated(got, basis, q)
    assert within(got, ref).all(), report(got, ref)
