"""Batched mixed-class path: Schwarz bounds on the device, screening,
CUDA-graph replay of a whole plan, and the autotuner's tier table."""
import numpy as np
import pytest

import oracle
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


def test_schwarz_bounds_match_oracle(eri):
    from paper_2605_10312_gb300 import screen
    basis = synth.water_cluster(2, seed=5)
    pairs, q = screen.pair_bounds(basis)
    diag = np.concatenate([pairs, pairs], axis=1)
    v, off = oracle.eri(basis, diag, nthreads=8)
    ref = np.empty(pairs.shape[0])
    ns = [1, 3, 5, 7, 9]
    for i, (a, b) in enumerate(pairs):
        n = ns[basis.shell_l[a]] * ns[basis.shell_l[b]]
        blk = v[off[i]:off[i + 1]].reshape(n, n)
        ref[i] = np.sqrt(np.max(np.abs(np.diag(blk))))
    np.testing.assert_allclose(q, ref, rtol=1e-10, atol=1e-14)


def test_screened_list_is_complete_and_bounded(eri):
    from paper_2605_10312_gb300 import screen
    basis = synth.water_cluster(3, seed=6)
    pairs, q = screen.pair_bounds(basis)
    thr = 1e-8
    got = synth.screened_quartets(q, pairs, thr)
    i, j = np.tril_indices(q.size)
    want = int(synth.survives(q[i], q[j], i, j, thr).sum())
    assert got.shape[0] == want
    # every dropped quartet is below the threshold: spot check by the oracle
    rng = np.random.default_rng(0)
    keep = {tuple(x) for x in got.tolist()}
    dropped = []
    while len(dropped) < 40:
        i, j = sorted(rng.integers(0, q.size, 2))[::-1]
        quad = (int(pairs[i][0]), int(pairs[i][1]), int(pairs[j][0]), int(pairs[j][1]))
        if q[i] * q[j] < thr and quad not in keep:
            dropped.append(quad)
    v, _ = oracle.eri(basis, np.array(dropped), nthreads=8)
    assert np.abs(v).max() <= thr * (1 + 1e-9)


def _canon(quartets, pairs):
    """Quartets -> set of (larger pair id, smaller pair id)."""
    pid = {(int(a), int(b)): k for k, (a, b) in enumerate(pairs)}
    out = set()
    for a, b, c, d in np.asarray(quartets).tolist():
        x, y = pid[(a, b)], pid[(c, d)]
        out.add((max(x, y), min(x, y)))
    return out


@pytest.mark.parametrize("thr", [1e-10, 1e-8, 1e-4])
def test_device_screening_matches_host(eri, thr):
    """The device survivor list (counting pass, prefix sum, compaction) is
    the host enumeration's set exactly, each unordered pair of pairs once,
    written as (larger pair index, smaller) in increasing order."""
    import torch
    from paper_2605_10312_gb300 import screen
    basis = synth.water_cluster(3, seed=6)
    pairs, qd = screen.pair_bounds_device(basis)
    q = qd.cpu().numpy()
    host = synth.screened_quartets(q, pairs, thr)
    dp = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).cuda()
    dev = eri.screen_quartets(qd.contiguous(), dp, thr).cpu().numpy()
    assert dev.shape == host.shape
    got = _canon(dev, pairs)
    assert len(got) == dev.shape[0] and got == _canon(host, pairs)
    pid = {(int(a), int(b)): k for k, (a, b) in enumerate(pairs)}
    order = [(pid[(a, b)], pid[(c, d)]) for a, b, c, d in dev.tolist()]
    assert all(x >= y for x, y in order) and order == sorted(order)
    # pairs sorted by falling bound: the host's list, element for element
    qs, ps = screen.sort_pairs(qd, dp)
    dev_sorted = eri.screen_quartets(qs, ps, thr).cpu().numpy()
    assert np.array_equal(dev_sorted, host)


def test_device_screening_edges(eri):
    """Threshold 0 keeps every unique quartet, an unreachable one none; a too
    small output is refused with the count still reported; no pairs, no
    quartets."""
    import ctypes
    import torch
    from paper_2605_10312_gb300 import screen
    basis = synth.water_cluster(1, seed=7)
    pairs, qd = screen.pair_bounds_device(basis)
    dp = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).cuda()
    n = pairs.shape[0]
    assert eri.screen_quartets(qd.contiguous(), dp, 0.0).shape == (n * (n + 1) // 2, 4)
    assert eri.screen_quartets(qd.contiguous(), dp, 1e300).shape == (0, 4)
    lib = eri.library()
    cnt = ctypes.c_int64()
    small = torch.empty((3, 4), dtype=torch.int32, device="cuda")
    rc = lib.eri_screen_quartets(qd.data_ptr(), dp.data_ptr(), n, 0.0, small.data_ptr(), 3, ctypes.byref(cnt), None)
    assert rc == -1 and cnt.value == n * (n + 1) // 2
    rc = lib.eri_screen_quartets(qd.data_ptr(), dp.data_ptr(), 0, 1e-10, None, 0, ctypes.byref(cnt), None)
    assert rc == 0 and cnt.value == 0


def test_graph_replay_and_parity(eri):
    import torch
    from paper_2605_10312_gb300 import screen
    basis = synth.water_cluster(3, seed=7)
    quartets = screen.screened(basis, threshold=1e-10)
    rng = np.random.default_rng(1)
    sample = quartets[rng.choice(quartets.shape[0], min(3000, quartets.shape[0]), replace=False)]
    p = eri.Plan(basis, sample)
    stream = torch.cuda.Stream()
    out = torch.empty(p.output_count, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        p.compute(out, stream)
        stream.synchronize()
        direct = out.cpu().numpy().copy()
        out.fill_(np.nan)
        p.capture(out, stream)
        p.replay(stream)
        stream.synchronize()
    replay = out.cpu().numpy()
    assert within(replay, direct, atol=1e-15, rtol=1e-13).all()
    ref, _ = adjudicated(direct, basis, sample)
    assert within(direct, ref).all(), report(direct, ref)
    p.close()


def test_autotune_keeps_results(eri):
    import torch
    from paper_2605_10312_gb300 import tune
    basis, q = synth.mixed_class_set([(1, 1, 0, 0), (2, 1, 1, 0), (2, 2, 2, 1)], 300, kset=(1, 3), seed=9)
    base = eri.eri(basis, q)[0].cpu().numpy()
    result = tune.autotune(basis, q, sample=256)
    assert result and all(v["tier"] in ("reg", "coop", "shared", "global") for v in result.values())
    tuned = eri.eri(basis, q)[0].cpu().numpy()
    assert within(tuned, base, atol=1e-14, rtol=1e-12).all()
    for c in result:
        eri.set_class_tier(c, 0)


def test_concurrent_lanes_match_serial(eri):
    """A mixed-class plan whose rounds run on several streams gives the same
    blocks as the serial plan (different classes write different blocks;
    chunked quartets reduce atomically into a zeroed block)."""
    import torch
    classes = [(1, 1, 0, 0), (2, 1, 1, 0), (2, 2, 1, 1), (3, 2, 2, 1), (3, 3, 3, 3), (4, 4, 2, 2)]
    basis, q = synth.mixed_class_set(classes, 200, kset=(1, 3, 6), seed=21)
    ps = eri.Plan(basis, q, streams=1)
    pc = eri.Plan(basis, q, streams=4)
    a = torch.empty(ps.output_count, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ps.compute(a, stream)
        pc.compute(b, stream)
        stream.synchronize()
        b2 = torch.empty_like(a)
        pc.capture(b2, stream)
        pc.replay(stream)
        stream.synchronize()
    assert within(b.cpu().numpy(), a.cpu().numpy(), atol=1e-15, rtol=1e-13).all()
    assert within(b2.cpu().numpy(), a.cpu().numpy(), atol=1e-15, rtol=1e-13).all()


def test_molecule_plans_match_plain_plans(eri):
    """Plans on a device-resident molecule (shared primitive-pair records,
    plan-local chunk aliases) give the blocks of ordinary plans, in FP64 and
    in mixed precision, with ordinary and stream-ordered memory."""
    import torch
    classes = [(1, 0, 0, 0), (2, 1, 1, 0), (2, 2, 1, 1), (3, 3, 2, 2), (4, 3, 2, 1)]
    basis, q = synth.mixed_class_set(classes, 150, kset=(1, 3, 6), seed=31)
    mol = eri.Mol(basis)
    stream = torch.cuda.Stream()
    qb = np.random.default_rng(0).uniform(0, 2e-6, q.shape[0])
    for kw in ({}, {"qbound": qb, "fp32_below": 1e-6}):
        pp = eri.Plan(basis, q, **kw)
        pm = eri.Plan(None, q, mol=mol, **kw)
        ps = eri.Plan(None, q, mol=mol, stream=stream, **kw)
        a = torch.empty(pp.output_count, dtype=torch.float64, device="cuda")
        b, c = torch.empty_like(a), torch.empty_like(a)
        with torch.cuda.stream(stream):
            pp.compute(a, stream)
            pm.compute(b, stream)
            ps.compute(c, stream)
            stream.synchronize()
        assert within(b.cpu().numpy(), a.cpu().numpy(), atol=1e-15, rtol=1e-13).all()
        assert within(c.cpu().numpy(), a.cpu().numpy(), atol=1e-15, rtol=1e-13).all()
        for p in (pp, pm, ps):
            p.close()
    mol.close()
