"""Coulomb/exchange digestion on the GPU against the oracle's J and K
(written out over the full ERI tensor)."""
import numpy as np
import pytest

import oracle
from paper_2605_10312_gb300 import synth
from ref import report, within

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eri():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_10312_gb300 import eri as m
    m.library()
    return m


def _density(nbf, seed):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((nbf, max(2, nbf // 3)))
    return C @ C.T / nbf


def _gpu_jk(eri, basis, quartets, D, via_blocks=True, persistent=False, tier="auto"):
    import torch
    p = eri.Plan(basis, quartets, digest=True, persistent=persistent, tier=tier)
    Dt = torch.from_numpy(D).cuda()
    J = torch.zeros_like(Dt)
    K = torch.zeros_like(Dt)
    if via_blocks:
        out = torch.empty(p.output_count, dtype=torch.float64, device="cuda")
        p.compute(out)
        p.digest_jk(out, Dt, J, K)
    else:
        p.compute_jk(Dt, J, K)
    torch.cuda.synchronize()
    return J.cpu().numpy(), K.cpu().numpy()


@pytest.mark.parametrize("via_blocks", [True, False])
def test_jk_tiny_set(eri, via_blocks):
    basis, _ = synth.tiny_set()
    q = synth.all_unique_quartets(basis.nshell)
    nbf = int(oracle.basis_function_offsets(basis)[-1])
    D = _density(nbf, 1)
    J, K = _gpu_jk(eri, basis, q, D, via_blocks=via_blocks)
    Jr, Kr = oracle.jk(basis, D, nthreads=8)
    assert within(J.ravel(), Jr.ravel()).all(), report(J.ravel(), Jr.ravel())
    assert within(K.ravel(), Kr.ravel()).all(), report(K.ravel(), Kr.ravel())


@pytest.mark.parametrize("via_blocks", [True, False])
def test_jk_water_any_representative(eri, via_blocks):
    """One water (O 3s 2p 1d, H 2s 1p): 12 shells, 24 functions.  Each orbit
    is passed through a random one of its 8 representatives."""
    basis = synth.water_cluster(1, seed=8)
    q = synth.all_unique_quartets(basis.nshell)
    rng = np.random.default_rng(2)
    perms = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2), (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]
    qr = np.array([row[list(perms[rng.integers(8)])] for row in q], dtype=np.int32)
    nbf = int(oracle.basis_function_offsets(basis)[-1])
    D = _density(nbf, 3)
    J, K = _gpu_jk(eri, basis, qr, D, via_blocks=via_blocks)
    Jr, Kr = oracle.jk(basis, D, nthreads=8)
    assert within(J.ravel(), Jr.ravel()).all(), report(J.ravel(), Jr.ravel())
    assert within(K.ravel(), Kr.ravel()).all(), report(K.ravel(), Kr.ravel())


def test_jk_graph_capture(eri):
    """eri_compute_jk and its captured graph (evaluation and digestion pass in
    one graph), replayed twice with J and K zeroed in between, against the
    oracle: two waters, every unique quartet (multi-part quartets in later
    part rounds, classes spread over several streams; the digestion lists
    are grouped by the launch that completes each quartet)."""
    import torch
    basis = synth.water_cluster(2, seed=8)
    q = synth.all_unique_quartets(basis.nshell)
    nbf = int(oracle.basis_function_offsets(basis)[-1])
    D = _density(nbf, 6)
    Jr, Kr = oracle.jk(basis, D, nthreads=8)
    p = eri.Plan(basis, q, digest=True)
    # some quartets have several parts (later part rounds add into them)
    assert sum(r["quartets"] for r in p.launches()[1:]) > q.shape[0]
    Dt = torch.from_numpy(D).cuda()
    J = torch.zeros_like(Dt)
    K = torch.zeros_like(Dt)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        p.compute_jk(Dt, J, K, st)
        st.synchronize()
        assert within(J.cpu().numpy().ravel(), Jr.ravel()).all()
        assert within(K.cpu().numpy().ravel(), Kr.ravel()).all()
        p.capture_jk(Dt, J, K, st)
        for _ in range(2):
            J.zero_()
            K.zero_()
            p.replay(st)
        st.synchronize()
    Jg, Kg = J.cpu().numpy(), K.cpu().numpy()
    assert within(Jg.ravel(), Jr.ravel()).all(), report(Jg.ravel(), Jr.ravel())
    assert within(Kg.ravel(), Kr.ravel()).all(), report(Kg.ravel(), Kr.ravel())


def test_jk_errors(eri):
    import torch
    basis, _ = synth.tiny_set()
    q = synth.all_unique_quartets(basis.nshell)
    p = eri.Plan(basis, q)
    D = torch.zeros((15, 15), dtype=torch.float64, device="cuda")
    J = torch.zeros_like(D)
    with pytest.raises(eri.EriError):
        p.compute_jk(D, J)
    p2 = eri.Plan(basis, q, digest=True)
    D2 = torch.zeros((14, 14), dtype=torch.float64, device="cuda")
    with pytest.raises(eri.EriError):
        p2.compute_jk(D2, torch.zeros_like(D2))


@pytest.mark.parametrize("nwater,tier", [(1, "auto"), (2, "auto"), (1, "coop")])
def test_jk_fused_into_persistent_launch(eri, nwater, tier):
    """A persistent digest plan digests each quartet inside the evaluation
    launch (the team finishing a quartet's last part; quartets whose parts
    all run on the register tier in a pass after it); J and K against the
    oracle's full-tensor contraction, for every unique quartet of one and two
    waters (multi-part quartets included), each orbit through a random
    representative.  tier "coop" puts every class in the persistent launch."""
    basis = synth.water_cluster(nwater, seed=8)
    q = synth.all_unique_quartets(basis.nshell)
    rng = np.random.default_rng(4)
    perms = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2), (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]
    qr = np.array([row[list(perms[rng.integers(8)])] for row in q], dtype=np.int32)
    nbf = int(oracle.basis_function_offsets(basis)[-1])
    D = _density(nbf, 5)
    J, K = _gpu_jk(eri, basis, qr, D, via_blocks=False, persistent=True, tier=tier)
    Jr, Kr = oracle.jk(basis, D, nthreads=8)
    assert within(J.ravel(), Jr.ravel()).all(), report(J.ravel(), Jr.ravel())
    assert within(K.ravel(), Kr.ravel()).all(), report(K.ravel(), Kr.ravel())
    # and the same as the separate digestion pass of an ordinary plan
    J2, K2 = _gpu_jk(eri, basis, qr, D, via_blocks=False)
    assert within(J.ravel(), J2.ravel(), atol=1e-13, rtol=1e-11).all()
    assert within(K.ravel(), K2.ravel(), atol=1e-13, rtol=1e-11).all()
