"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times (the same plans over the same seeded quartet lists), on
sampled quartets the oracle evaluates one by one; and the largest
contraction depth the ABI accepts."""
import numpy as np
import pytest

import bench
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


@pytest.mark.parametrize("k", range(len(bench.SWEEP)))
def test_benchmark_workload_sampled(eri, k):
    import torch
    ls, n = bench.SWEEP[k]
    basis, q = synth.class_sweep(ls, n, kset=bench.KSET, seed=bench.SEED + 10 * ls[0])
    p = eri.Plan(basis, q)
    out = torch.empty(p.output_count, dtype=torch.float64, device="cuda")
    p.compute(out)
    torch.cuda.synchronize()
    off = p.offsets()
    rng = np.random.default_rng(7 + k)
    m = {1: 400, 2: 120, 3: 24, 4: 8}[ls[0]]
    # the first and last quartets, and a seeded sample in between
    pick = np.unique(np.concatenate([[0, n - 1], rng.choice(n, m, replace=False)]))
    got = np.concatenate([out[off[i]:off[i + 1]].cpu().numpy() for i in pick])
    ref, _ = adjudicated(got, basis, q[pick], nthreads=16)
    assert within(got, ref).all(), report(got, ref)
    p.close()


def test_largest_contraction_depth(eri):
    """K = 32 primitives per shell (the ABI's maximum): 32^4 primitive
    quartets per shell quartet, chunked across teams or lanes."""
    from paper_2605_10312_gb300.eri import Plan  # noqa: F401
    for ls in ((1, 0, 0, 0), (2, 1, 1, 0)):
        basis, q = synth.class_sweep(ls, 3, kset=(32,), seed=90 + ls[0], box_angstrom=3.0)
        import torch
        p = eri.Plan(basis, q)
        out = torch.empty(p.output_count, dtype=torch.float64, device="cuda")
        p.compute(out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref, _ = adjudicated(got, basis, q, nthreads=16)
        assert within(got, ref).all(), (ls, report(got, ref))
