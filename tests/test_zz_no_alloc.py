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


@pytest.mark.parametrize("ls,n,kset", [((2, 2, 1, 0), 300, (1, 2, 3)), ((3, 2, 2, 1), 200, (1, 2)),
                                       ((4, 4, 4, 4), 3, (1, 2))])
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
        p.compute_fixed_scratch(got)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        assert np.isfinite(got).all(), call
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
