"""Mixed precision: quartets whose Schwarz bound is below the threshold run
their recurrences in FP32; the rest, and every store, stay FP64.  The mixed
plan must agree with the all-FP64 plan within 1e-10 absolute, and its FP64
quartets must be identical to the FP64 plan's."""
import numpy as np
import pytest

from paper_2605_10312_gb300 import synth
from ref import adjudicated, blocks, report, within

pytestmark = pytest.mark.gpu

FP32_BELOW = 1e-6
MIXED_ATOL = 1e-10


@pytest.fixture(scope="module")
def eri():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_10312_gb300 import eri as m
    m.library()
    return m


def _quartet_bounds(basis, quartets):
    from paper_2605_10312_gb300 import screen
    pairs, q = screen.pair_bounds(basis)
    index = {tuple(p): k for k, p in enumerate(pairs.tolist())}

    def qp(a, b):
        return q[index[(a, b) if a >= b else (b, a)]]
    return np.array([qp(a, b) * qp(c, d) for a, b, c, d in quartets.tolist()])


def _cluster_sample(nwater, layout, seed, n):
    from paper_2605_10312_gb300 import screen
    basis = synth.water_cluster(nwater, seed=seed, layout=layout)
    quartets = screen.screened(basis, threshold=1e-12)
    rng = np.random.default_rng(seed)
    qb = _quartet_bounds(basis, quartets)
    # half below the FP32 threshold, half above (as far as available)
    lo, hi = np.flatnonzero(qb < FP32_BELOW), np.flatnonzero(qb >= FP32_BELOW)
    pick = np.concatenate([rng.choice(lo, min(n // 2, lo.size), replace=False),
                           rng.choice(hi, min(n // 2, hi.size), replace=False)])
    rng.shuffle(pick)
    return basis, quartets[pick], qb[pick]


@pytest.mark.parametrize("layout,nwater", [("dz", 4), ("tz", 3)])
def test_mixed_matches_fp64(eri, layout, nwater):
    import torch
    basis, q, qb = _cluster_sample(nwater, layout, seed=11, n=6000)
    assert (qb < FP32_BELOW).sum() > 500
    p64 = eri.Plan(basis, q)
    pmx = eri.Plan(basis, q, qbound=qb, fp32_below=FP32_BELOW)
    st = pmx.stats()
    assert st["fp32_parts"] > 0 and st["flops_fp32"] > 0
    a = torch.empty(p64.output_count, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    p64.compute(a)
    pmx.set_timing(True)
    pmx.compute(b)
    torch.cuda.synchronize()
    assert any(r["precision"] == 32 for r in pmx.launches()[1:])
    a, b = a.cpu().numpy(), b.cpu().numpy()
    off = p64.offsets()
    fp32 = np.repeat(qb < FP32_BELOW, np.diff(off))
    d = np.abs(a - b)
    assert d[~fp32].max(initial=0) <= 1e-13 * max(1.0, np.abs(a[~fp32]).max(initial=0)), "FP64 quartets changed"
    assert d[fp32].max() <= MIXED_ATOL, d[fp32].max()
    # and each quartet's error stays within a small multiple of its bound x 2^-24
    per_q = np.maximum.reduceat(d, off[:-1]) if d.size else d
    assert (per_q <= 64 * 2.0 ** -24 * qb + 1e-36).all()
    # the FP64 part against the oracle
    sel = np.flatnonzero(qb >= FP32_BELOW)[:400]
    ref, _ = adjudicated(np.concatenate([b[off[i]:off[i + 1]] for i in sel]), basis, q[sel])
    got = np.concatenate([b[off[i]:off[i + 1]] for i in sel])
    assert within(got, ref).all(), report(got, ref)


def test_mixed_threshold_zero_is_fp64(eri):
    import torch
    basis, q = synth.class_sweep((2, 1, 1, 0), 300, kset=(1, 3), seed=2)
    qb = np.full(q.shape[0], 1e-3)
    # ordered: parts add in a fixed order, so the two agree bit for bit
    p64 = eri.Plan(basis, q, ordered=True)
    pmx = eri.Plan(basis, q, qbound=qb, fp32_below=0.0, ordered=True)
    assert pmx.stats()["fp32_parts"] == 0
    a = torch.empty(p64.output_count, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    p64.compute(a)
    pmx.compute(b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_mixed_all_fp32_every_tier_class(eri):
    """Every class in FP32 form (register and cooperative) against the oracle
    with a tolerance scaled by the block's magnitude."""
    import torch
    classes = [(1, 1, 1, 1), (2, 2, 1, 0), (2, 2, 2, 1), (3, 3, 2, 2), (3, 3, 3, 3)]
    basis, q = synth.mixed_class_set(classes, 40, kset=(1, 3), seed=5)
    # exact Schwarz bounds from the oracle's (ab|ab) blocks
    pairs = np.unique(np.concatenate([q[:, :2], q[:, 2:]]), axis=0)
    diag, doff = blocks(basis, np.concatenate([pairs, pairs], axis=1))
    qpair = {tuple(pr): np.sqrt(np.abs(diag[doff[k]:doff[k + 1]]).max()) for k, pr in enumerate(pairs.tolist())}
    qb = np.array([qpair[(a, b)] * qpair[(c, d)] for a, b, c, d in q.tolist()])
    p = eri.Plan(basis, q, qbound=qb, fp32_below=1e300)
    assert p.stats()["fp32_parts"] > 0
    out = torch.empty(p.output_count, dtype=torch.float64, device="cuda")
    p.compute(out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref, off = blocks(basis, q, long_double=True)
    for i in range(q.shape[0]):
        g, r = got[off[i]:off[i + 1]], ref[off[i]:off[i + 1]]
        # FP32 recurrences: error a small multiple of 2^-24 times the bound,
        # plus the FP32 underflow floor (values below ~1e-38 are not normal)
        assert np.abs(g - r).max() <= 64 * 2.0 ** -24 * qb[i] + 1e-36, (q[i], np.abs(g - r).max(), qb[i])


def test_mixed_bad_arguments(eri):
    basis, q = synth.class_sweep((1, 0, 0, 0), 10, seed=1)
    with pytest.raises(eri.EriError):
        eri.Plan(basis, q, qbound=-np.ones(q.shape[0]), fp32_below=1e-6)
    with pytest.raises(eri.EriError):
        eri.Plan(basis, q, qbound=np.ones(q.shape[0]), fp32_below=float("inf"))
    with pytest.raises(ValueError):
        eri.Plan(basis, q, qbound=np.ones(3), fp32_below=1e-6)


def test_mixed_error_vs_oracle_per_class(eri):
    """The mixed-precision workload's layout (tz water cluster, Schwarz 1e-10,
    FP32 below 1e-6) on a seeded sample of its screened list, against the
    FP64 oracle (long-double adjudicated): every element within 1e-10
    absolute, per class; the per-class max and RMS errors are printed (run
    with -s)."""
    import torch
    from paper_2605_10312_gb300 import screen
    basis = synth.water_cluster(5, seed=3, layout="tz")
    pairs, qp = screen.pair_bounds(basis)
    q = synth.sample_screened_quartets(qp, pairs, 1e-10, 3000, seed=7)
    qb = screen.quartet_bounds(qp, q)
    assert (qb < FP32_BELOW).sum() > 1000
    p = eri.Plan(basis, q, qbound=qb, fp32_below=FP32_BELOW)
    out = torch.empty(p.output_count, dtype=torch.float64, device="cuda")
    p.compute(out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref, off = adjudicated(got, basis, q)
    d = np.abs(got - ref)
    ls = basis.shell_l[q]
    labels = np.array(["".join("spdfg"[x] for x in row) for row in ls])
    elem_label = np.repeat(labels, np.diff(off))
    elem_fp32 = np.repeat(qb < FP32_BELOW, np.diff(off))
    worst = 0.0
    for lab in sorted(set(labels)):
        m = elem_label == lab
        mx, rms = d[m].max(), float(np.sqrt(np.mean(d[m] ** 2)))
        worst = max(worst, mx)
        print("class {} quartets {} fp32 {} max|d| {:.3g} rms {:.3g}".format(
            lab, int((labels == lab).sum()), int((m & elem_fp32).sum()), mx, rms))
    assert worst <= MIXED_ATOL, worst
