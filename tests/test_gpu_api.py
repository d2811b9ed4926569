"""Boundary behaviour of the CUDA path: host-buffer entry point, offsets,
empty plans, tier routing and forced tiers."""
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


def test_compute_host_matches_device(eri):
    import torch
    basis, q = synth.class_sweep((2, 1, 1, 0), 500, kset=(1, 3), seed=9, box_angstrom=3.0)
    # ordered: parts add in a fixed order, so two evaluations agree bit for bit
    p = eri.Plan(basis, q, ordered=True)
    dev = torch.empty(p.output_count, dtype=torch.float64, device="cuda")
    p.compute(dev)
    host = torch.empty(p.output_count, dtype=torch.float64).pin_memory()
    p.compute_host(host)
    torch.cuda.synchronize()
    assert torch.equal(dev.cpu(), host)
    p.close()


def test_empty_plan(eri):
    import torch
    basis, _ = synth.tiny_set()
    p = eri.Plan(basis, np.zeros((0, 4), dtype=np.int32))
    assert p.output_count == 0
    p.compute(torch.empty(1, dtype=torch.float64, device="cuda"))
    p.close()


@pytest.mark.parametrize("tier,ls", [("reg", (1, 1, 1, 0)), ("shared", (1, 1, 1, 0)), ("global", (1, 1, 1, 0)),
                                     ("shared", (2, 2, 1, 0)), ("shared", (3, 1, 1, 0)), ("global", (2, 2, 1, 1)),
                                     ("global", (3, 2, 2, 1)), ("coop", (2, 2, 2, 1)), ("coop", (3, 3, 2, 2))])
def test_forced_tiers_agree(eri, tier, ls):
    """The same class through each tier that can hold it gives the oracle's
    values (register tier only for the classes compiled straight-line)."""
    basis, q = synth.class_sweep(ls, 300, kset=(1, 2, 3), seed=19, box_angstrom=3.0)
    for t in (tier, "auto"):
        got = eri.eri(basis, q, tier=t)[0].cpu().numpy()
        ref, _ = adjudicated(got, basis, q)
        assert within(got, ref).all(), (t, report(got, ref))


def test_orientation_option(eri):
    """Higher-l-first orientation is also correct on a compact geometry."""
    basis, q = synth.class_sweep((2, 2, 1, 1), 100, kset=(1, 2), seed=23, box_angstrom=2.0, exp_range=(0.2, 10.0))
    got = eri.eri(basis, q, orientation="l")[0].cpu().numpy()
    ref, _ = adjudicated(got, basis, q)
    assert within(got, ref).all(), report(got, ref)


def test_unsupported_tier_is_an_error(eri):
    basis, q = synth.class_sweep((4, 4, 4, 4), 2, seed=3)
    with pytest.raises(eri.EriError) as e:
        eri.Plan(basis, q, tier="reg")
    assert e.value.code == -2


def test_ordered_parts_and_one_round_agree(eri):
    """The default plan runs every part of a multi-part quartet in one launch
    round, reducing into the zeroed block; an ordered plan adds the parts in
    round order.  Same blocks up to the order of the additions, fewer launches
    by default, and the ordered plan is bitwise reproducible."""
    import torch
    basis = synth.water_cluster(2, seed=8)
    q = synth.all_unique_quartets(basis.nshell)
    p1 = eri.Plan(basis, q)
    p2 = eri.Plan(basis, q, ordered=True)
    assert p1.stats()["launches"] < p2.stats()["launches"]
    a = torch.empty(p1.output_count, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    p1.compute(a)
    p2.compute(b)
    p2.compute(c)
    torch.cuda.synchronize()
    assert torch.equal(b, c)
    assert torch.allclose(a, b, rtol=1e-13, atol=1e-16)
    with pytest.raises(eri.EriError):
        eri.Plan(basis, q, ordered=True, persistent=True)
