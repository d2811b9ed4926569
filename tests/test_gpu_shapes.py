"""Every team-cooperative shape the build ships for a class (the deep and
shallow choices and the autotuner's alternatives, eri_class_shapes), with
the optional FP64 terms predicated and behind warp votes, installed for all
three kinds of contraction (eri_set_class_shape) and compared with the CPU
oracle element by element within |d| <= max(1e-12, 1e-10 |ref|).  The
contraction depths K per shell from {1, 1, 1, 2, 3} give deep, shallow and
single-primitive parts in one plan; the launch records must show the shape
installed.  Also a persistent plan (the work list takes each item's shape
from its bucket) and the autotuner itself on a small mixed set."""
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


CLASSES = {(2, 2, 2, 2): 24, (3, 3, 2, 2): 8, (3, 2, 2, 1): 16, (4, 4, 3, 3): 3}


def _case(ls, seed):
    # whole pairs on the higher l keep every part in the class itself
    return synth.class_sweep(ls, CLASSES[ls], kset=(1, 1, 1, 2, 3), seed=seed, box_angstrom=2.0,
                             exp_range=(0.2, 10.0))


def _set_all(eri, ls, shape, votes):
    for kind in eri.KINDS:
        eri.set_class_shape(ls, kind, shape, votes)


@pytest.mark.parametrize("ls", list(CLASSES))
def test_every_shipped_shape_matches_oracle(eri, ls):
    basis, q = _case(ls, 4700 + sum(ls))
    shapes = eri.class_shapes(ls)
    assert len(shapes) >= 2
    ref = None
    try:
        for i, shp in enumerate(shapes):
            for votes in ("off", "on"):
                _set_all(eri, ls, i, votes)
                import torch
                p = eri.Plan(basis, q, orientation="l", tier="coop")
                out = torch.full((p.output_count,), float("nan"), dtype=torch.float64, device="cuda")
                p.set_timing(True)
                p.compute(out)
                torch.cuda.synchronize()
                recs = [r for r in p.launches()[1:] if r["tier"] == 4]
                assert recs and all(r["shape"] == i and r["team"] == shp["T"] and r["votes"] == votes for r in recs)
                got = out.cpu().numpy()
                p.close()
                if ref is None:
                    ref, _ = adjudicated(got, basis, q)
                assert within(got, ref).all(), (i, votes, report(got, ref))
    finally:
        _set_all(eri, ls, -1, "auto")


def test_persistent_plan_takes_the_installed_shape(eri):
    import torch
    ls = (3, 3, 2, 2)
    basis, q = _case(ls, 4800)
    shapes = eri.class_shapes(ls)
    try:
        _set_all(eri, ls, len(shapes) - 1, "on")
        got, _ = eri.eri(basis, q, orientation="l", persistent=True, tier="coop")
        got = got.cpu().numpy()
    finally:
        _set_all(eri, ls, -1, "auto")
    ref, _ = adjudicated(got, basis, q)
    assert within(got, ref).all(), report(got, ref)


def test_autotuned_plan_matches_oracle(eri):
    """The autotuner (tiers, then shapes and vote forms per kind) on a mixed
    set; a plan built under its choices against the oracle."""
    from paper_2605_10312_gb300 import tune
    sets = [_case(ls, 4900 + sum(ls)) for ls in ((2, 2, 2, 2), (3, 2, 2, 1))]
    basis, q = synth.concat_sets(sets, shuffle_seed=5)
    res = tune.autotune(basis, q, sample=64, reps=1, shapes=True)
    try:
        assert any("shapes" in v for v in res.values())
        got, _ = eri.eri(basis, q, orientation="l")
        got = got.cpu().numpy()
        ref, _ = adjudicated(got, basis, q)
        assert within(got, ref).all(), report(got, ref)
    finally:
        for c in res:
            eri.set_class_tier(c, 0)
            for kind in eri.KINDS:
                eri.set_class_shape(c, kind, -1)
