"""Persistent plans (eri_opts.persistent): the cooperative classes of a plan
(with tier "coop": every class) in one launch per precision and vote form
over a device work list, the compiled register-tier classes in their own
launches, the parts of a quartet reduced into its zeroed block.

Against the oracle element by element within |d| <= max(1e-12, 1e-10 |ref|):
the tiny s/p set (every class of it, quartets split into up to four oriented
parts), a mixed-class set with deep and single-primitive contractions
through (gg|gg), a screened water cluster (also against the per-bucket plan
and through CUDA-graph replay), molecule plans, and mixed precision (the
FP32 quartets within their bound)."""
import numpy as np
import pytest

from paper_2605_10312_gb300 import synth
from ref import adjudicated, blocks, report, within

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eri():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_10312_gb300 import eri as m
    m.library()
    return m


def _compute(eri, basis, q, **opts):
    import torch
    p = eri.Plan(basis, q, **opts)
    out = torch.full((max(1, p.output_count),), float("nan"), dtype=torch.float64, device="cuda")
    p.set_timing(True)
    p.compute(out)
    torch.cuda.synchronize()
    launches = p.launches()
    off = p.offsets()
    p.close()
    return out.cpu().numpy()[:off[-1]], off, launches


@pytest.mark.parametrize("tier", ["auto", "coop"])
def test_tiny_set_persistent(eri, tier):
    """tier "auto": the s/p classes keep their compiled kernels (their parts
    reduce into zeroed blocks too); tier "coop": everything on the work
    list."""
    basis, q = synth.tiny_set(seed=1)
    got, off, launches = _compute(eri, basis, q, persistent=True, tier=tier)
    assert all(l["tier"] == (5 if tier == "coop" else 1) for l in launches[1:])
    ref, roff = adjudicated(got, basis, q)
    assert np.array_equal(off, roff)
    assert within(got, ref).all(), report(got, ref)


def test_mixed_classes_persistent(eri):
    """With tier "coop" the register-tier classes run on their cooperative
    programs too; deep contractions (K = 6, chunked) and single-primitive
    parts reduce into zeroed blocks with the other parts of their quartet."""
    classes = [(0, 0, 0, 0), (1, 0, 1, 0), (1, 1, 1, 1), (2, 1, 1, 0), (2, 2, 2, 1), (3, 2, 2, 1), (3, 3, 3, 3),
               (4, 4, 2, 2), (4, 4, 4, 4)]
    parts = [synth.class_sweep(ls, {0: 60, 1: 40, 2: 20, 3: 8, 4: 3}[max(ls)],
                               kset=(1, 2, 6) if max(ls) < 4 else (1, 2), seed=600 + i, box_angstrom=3.0,
                               exp_range=(0.1, 60.0)) for i, ls in enumerate(classes)]
    basis, q = synth.concat_sets(parts, shuffle_seed=3)
    got, _, launches = _compute(eri, basis, q, persistent=True, tier="coop")
    assert len(launches) <= 1 + 2  # pair set-up, then one launch per vote form
    ref, _ = adjudicated(got, basis, q)
    assert within(got, ref).all(), report(got, ref)
    # register-tier classes on their compiled kernels, the rest persistent
    got, _, launches = _compute(eri, basis, q, persistent=True)
    assert sum(1 for l in launches[1:] if l["tier"] == 5) <= 2
    ref, _ = adjudicated(got, basis, q)
    assert within(got, ref).all(), report(got, ref)


def test_water_cluster_persistent_matches_buckets_and_replays(eri):
    import torch
    from paper_2605_10312_gb300 import screen
    basis = synth.water_cluster(4, seed=7)
    quartets = screen.screened(basis, threshold=1e-10)
    rng = np.random.default_rng(2)
    sample = quartets[rng.choice(quartets.shape[0], min(6000, quartets.shape[0]), replace=False)]
    pb = eri.Plan(basis, sample)
    pp = eri.Plan(basis, sample, persistent=True)
    a = torch.empty(pb.output_count, dtype=torch.float64, device="cuda")
    b = torch.full_like(a, float("nan"))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pb.compute(a, stream)
        pp.compute(b, stream)
        stream.synchronize()
        c = torch.full_like(a, float("nan"))
        pp.capture(c, stream)
        pp.replay(stream)
        pp.replay(stream)
        stream.synchronize()
    a, b, c = a.cpu().numpy(), b.cpu().numpy(), c.cpu().numpy()
    assert within(b, a, atol=1e-15, rtol=1e-13).all()
    assert within(c, b, atol=1e-15, rtol=1e-13).all()
    sel = rng.choice(sample.shape[0], 1500, replace=False)
    off = pp.offsets()
    got = np.concatenate([b[off[i]:off[i + 1]] for i in sel])
    ref, _ = adjudicated(got, basis, sample[sel])
    assert within(got, ref).all(), report(got, ref)
    pb.close()
    pp.close()


def test_molecule_plan_persistent(eri):
    classes = [(1, 0, 0, 0), (2, 1, 1, 0), (2, 2, 1, 1), (3, 3, 2, 2), (4, 3, 2, 1)]
    basis, q = synth.mixed_class_set(classes, 60, kset=(1, 3, 6), seed=31)
    mol = eri.Mol(basis)
    got, _, _ = _compute(eri, None, q, mol=mol, persistent=True)
    ref, _ = adjudicated(got, basis, q)
    assert within(got, ref).all(), report(got, ref)
    mol.close()


def test_mixed_precision_persistent(eri):
    """FP32 quartets of a persistent plan (their own launch) within a small
    multiple of 2^-24 times their bound of the long-double oracle; FP64
    quartets within the FP64 tolerance."""
    classes = [(1, 1, 1, 1), (2, 2, 1, 0), (2, 2, 2, 1), (3, 3, 2, 2)]
    basis, q = synth.mixed_class_set(classes, 40, kset=(1, 3), seed=5)
    pairs = np.unique(np.concatenate([q[:, :2], q[:, 2:]]), axis=0)
    diag, doff = blocks(basis, np.concatenate([pairs, pairs], axis=1))
    qpair = {tuple(pr): np.sqrt(np.abs(diag[doff[k]:doff[k + 1]]).max()) for k, pr in enumerate(pairs.tolist())}
    qb = np.array([qpair[(a, b)] * qpair[(c, d)] for a, b, c, d in q.tolist()])
    thr = float(np.median(qb))
    got, off, launches = _compute(eri, basis, q, qbound=qb, fp32_below=thr, persistent=True)
    assert any(l["precision"] == 32 for l in launches[1:])
    ref, roff = blocks(basis, q, long_double=True)
    for i in range(q.shape[0]):
        g, r = got[off[i]:off[i + 1]], ref[roff[i]:roff[i + 1]]
        if qb[i] < thr:
            assert np.abs(g - r).max() <= 64 * 2.0 ** -24 * qb[i] + 1e-36, (q[i], np.abs(g - r).max(), qb[i])
        else:
            assert within(g, r).all(), (q[i], report(g, r))


def test_persistent_rejects_other_tiers(eri):
    basis, q = synth.class_sweep((1, 1, 1, 1), 10, seed=3)
    with pytest.raises(eri.EriError) as e:
        eri.Plan(basis, q, tier="reg", persistent=True)
    assert e.value.code == -1
