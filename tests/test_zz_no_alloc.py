"""The allocation-free entry point eri_compute_fixed_scratch.

Callers that cannot allocate device memory while they evaluate (a
device-memory budget owned by another framework, or a latency-critical loop
that must not enter the allocator, which can synchronise the device) use this
variant of the global-scratch executor, whose per-thread value slots live in a
fixed device array the library holds.  It must give the same integrals as
eri_compute on the same plan, on two calls in a row (the array keeps the
previous call's contents)."""
import numpy as np
import pytest

from paper_2605_10312_gb300 import synth
from ref import within

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eri():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_10312_gb300 import eri as m
    m.library()
    return m


# (gg|gg) with 130 quartets: the plan's grid has two 128-thread blocks, the
# fixed array holds one (41 MB per block), so that block strides over the
# quartets beyond its 128 threads
@pytest.mark.parametrize("ls,n,kset", [((2, 2, 1, 0), 300, (1, 2, 3)), ((3, 2, 2, 1), 200, (1, 2)),
                                       ((4, 4, 4, 4), 3, (1, 2)), ((4, 4, 4, 4), 130, (1,))])
def test_fixed_scratch_matches_compute(eri, ls, n, kset):
    import torch
    basis, q = synth.class_sweep(ls, n, kset=kset, seed=71, box_angstrom=3.0)
    p = eri.Plan(basis, q, tier="global")
    ref = torch.empty(p.output_count, dtype=torch.float64, device="cuda")
    p.compute(ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    for call in range(2):
        got = torch.full((p.output_count,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        p.compute_fixed_scratch(got)
        torch.cuda.synchronize()
        if call == 1:
            # the second call finds everything in place: no device memory
            # changes hands (the first call may still look up the array)
            assert torch.cuda.mem_get_info()[0] == free0
        got = got.cpu().numpy()
        assert np.isfinite(got).all(), call
        assert within(got, ref).all(), (call, np.abs(got - ref).max())
    p.close()


def test_fixed_scratch_deep_contraction_on_a_tuned_tier(eri):
    """A class the autotuner sends to the global-scratch tier is never cut
    into chunks that reduce into their block (only the cooperative tier
    reduces chunks): a deep contraction (K = 6, 1296 primitive quartets)
    gives the oracle's blocks through eri_compute and through the
    allocation-free entry point, twice in a row."""
    import torch
    from ref import adjudicated
    ls = (3, 2, 2, 1)
    # whole pairs on the higher l: every part of every quartet is of class ls
    basis, q = synth.class_sweep(ls, 40, kset=(6,), seed=72, box_angstrom=2.0, exp_range=(0.2, 10.0))
    eri.set_class_tier(ls, "global")
    try:
        p = eri.Plan(basis, q, orientation="l")
    finally:
        eri.set_class_tier(ls, 0)
    ref = eri.eri(basis, q, tier="coop", orientation="l")[0].cpu().numpy()
    ref, _ = adjudicated(ref, basis, q)
    assert [l["tier"] for l in p.launches()[1:]] == [3] * (len(p.launches()) - 1)
    for call in range(3):
        got = torch.full((p.output_count,), float("nan"), dtype=torch.float64, device="cuda")
        if call == 0:
            p.compute(got)
        else:
            p.compute_fixed_scratch(got)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        assert within(got, ref).all(), (call, np.abs(got - ref).max())
    p.close()


def test_fixed_scratch_rejects_other_tiers(eri):
    import torch
    basis, q = synth.class_sweep((1, 1, 1, 1), 10, seed=3)
    p = eri.Plan(basis, q)  # register tier
    out = torch.empty(p.output_count, dtype=torch.float64, device="cuda")
    with pytest.raises(eri.EriError) as e:
        p.compute_fixed_scratch(out)
    assert e.value.code == -2
    p.close()
