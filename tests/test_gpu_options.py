"""GPU parity of every option path the C ABI exposes, and of the device Boys
function on its own.

The paper's ablations (Sec. V-B) switch the axis rule (Algorithm 1 as
printed, or the common bra-first x->y->z order, instead of the prose reading),
the DSA order (Eq. 7) for a level order, and the spherical fusion (Eq. 16)
for materialize-then-transform (Eq. 17) or Cartesian output.  Each of these
generated programs is compared here with the CPU oracle element by element
within |d| <= max(1e-12, 1e-10 |ref|), on every class the library builds
the variants for, on the cooperative tier (what tier 0 routes them to) and
on the thread-per-quartet global-scratch tier.  So are the two whole-pair
orientations, the (gg|gg) class on the global-scratch tier, and the identity
stepwise == materialize on the same plan (the Eq. 14 identity, GPU against
GPU)."""
import numpy as np
import pytest

import oracle
from paper_2605_10312_gb300 import synth
from paper_2605_10312_gb300.build import ABLATION_CLASSES, ABLATION_OPTS
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


# quartets per class: enough to fill several teams, small enough for the oracle
NQ = {(1, 1, 1, 1): 160, (2, 1, 2, 1): 100, (2, 2, 2, 1): 60, (2, 2, 2, 2): 30, (3, 3, 2, 2): 8, (3, 3, 3, 3): 4}
OPT_IDS = ["-".join(o) for o in ABLATION_OPTS]


def _case(ls, seed):
    # compact geometry with mixed exponents: integrals up to order one, where
    # the absolute floor of the tolerance hides nothing; exponents within a
    # factor 50, so that whole-pair orientation keeps HRR within tolerance
    return synth.class_sweep(ls, NQ[ls], kset=(1, 2, 3), seed=seed, box_angstrom=2.0, exp_range=(0.2, 10.0))


def _opts(o):
    # the variants are generated for the classes in their canonical order
    # (la >= lb, lc >= ld): whole pairs recur on the higher l, so every part
    # stays in its class
    axis, sched, sph = o
    return dict(axis_rule=axis, schedule=sched, sph_mode=sph, orientation="l")


@pytest.mark.parametrize("opt", ABLATION_OPTS, ids=OPT_IDS)
@pytest.mark.parametrize("ls", ABLATION_CLASSES)
def test_ablation_variant_matches_oracle(eri, ls, opt):
    """Each ablation program (cooperative tier under tier 0) against the
    oracle; Cartesian output against the oracle's Cartesian blocks."""
    basis, q = _case(ls, 4100 + sum(ls))
    got, off = eri.eri(basis, q, **_opts(opt))
    got = got.cpu().numpy()
    ref, roff = adjudicated(got, basis, q, cart=opt[2] == "cart")
    assert np.array_equal(off, roff)
    assert within(got, ref).all(), report(got, ref)


@pytest.mark.parametrize("opt", ABLATION_OPTS, ids=OPT_IDS)
@pytest.mark.parametrize("ls", [(2, 1, 2, 1), (2, 2, 2, 1)])
def test_ablation_variant_global_tier(eri, ls, opt):
    """The same variants through the thread-per-quartet program tier."""
    basis, q = _case(ls, 4200 + sum(ls))
    got, _ = eri.eri(basis, q, tier="global", **_opts(opt))
    got = got.cpu().numpy()
    ref, _ = adjudicated(got, basis, q, cart=opt[2] == "cart")
    assert within(got, ref).all(), report(got, ref)


@pytest.mark.parametrize("ls", ABLATION_CLASSES)
def test_stepwise_equals_materialize_on_gpu(eri, ls):
    """Eq. 16 (stepwise) and Eq. 17 (materialize) give the same blocks on the
    same plan input (GPU against GPU)."""
    basis, q = _case(ls, 4300 + sum(ls))
    a = eri.eri(basis, q, sph_mode="stepwise", orientation="l")[0].cpu().numpy()
    b = eri.eri(basis, q, sph_mode="materialize", orientation="l")[0].cpu().numpy()
    assert within(b, a).all(), report(b, a)


@pytest.mark.parametrize("orientation", ["l", "tight"])
@pytest.mark.parametrize("ls", [(1, 1, 1, 0), (2, 2, 1, 1), (3, 2, 2, 1), (3, 3, 2, 2), (4, 2, 3, 1)])
def test_whole_pair_orientations(eri, ls, orientation):
    """Orientation 1 (whole pair on the higher l) and 2 (on the shell with the
    largest exponent), on a compact geometry with exponents in [0.2, 10]
    (mixed enough that the orientations differ, narrow enough that a
    whole-pair orientation keeps HRR within the tolerance)."""
    n = {0: 120, 1: 120, 2: 60, 3: 12, 4: 8}[max(ls)]
    basis, q = synth.class_sweep(ls, n, kset=(1, 2), seed=4400 + sum(ls), box_angstrom=2.0, exp_range=(0.2, 10.0))
    got = eri.eri(basis, q, orientation=orientation)[0].cpu().numpy()
    ref, _ = adjudicated(got, basis, q)
    assert within(got, ref).all(), report(got, ref)


def test_gggg_global_tier(eri):
    """(gg|gg) on the thread-per-quartet global-scratch tier against the
    oracle (the allocation-free entry point runs this tier)."""
    basis, q = synth.class_sweep((4, 4, 4, 4), 3, kset=(1, 2), seed=4500, box_angstrom=3.0, exp_range=(0.1, 60.0))
    got = eri.eri(basis, q, tier="global")[0].cpu().numpy()
    ref, _ = adjudicated(got, basis, q)
    assert within(got, ref).all(), report(got, ref)


def _boys_args():
    """Seeded arguments over the whole range the path meets (T up to about
    3e5 on the 10 Angstrom sweep geometry): log-uniform, uniform below the
    table edge, the table's grid points and midpoints, both sides of the
    switch to the asymptotic branch at T = 36, and T = 0."""
    rng = np.random.default_rng(4600)
    parts = [np.zeros(1), 10.0 ** rng.uniform(-12, np.log10(3e5), 600), rng.uniform(0, 36, 600),
             np.arange(0, 361) * 0.1, np.arange(0, 360) * 0.1 + 0.05,
             36.0 + np.array([-1e-9, -1e-12, 0.0, 1e-12, 1e-9]), rng.uniform(35.5, 36.5, 200),
             rng.uniform(36, 60, 200)]
    return np.concatenate(parts)


@pytest.mark.parametrize("form", ["reg", "coop", "exec"])
def test_device_boys(eri, form):
    """F_m(T), m = 0..16, of each tier's device routine against the oracle's
    long-double Boys function (series and downward recursion, erf and upward
    recursion above T = 50; pinned to mpmath quadrature): relative error at
    most 1e-13 for every m and T.  Also for lower orders L (the downward
    recursion starts at F_L)."""
    import torch
    T = _boys_args()
    Td = torch.tensor(T, dtype=torch.float64, device="cuda")
    for L in (16, 9, 4, 0):
        F = eri.boys(Td, L, form=form).cpu().numpy()
        ref = np.array([oracle.boys(L, t, long_double=True) for t in T])
        rel = np.abs(F - ref) / np.maximum(np.abs(ref), 1e-300)
        worst = np.unravel_index(np.argmax(rel), rel.shape)
        assert rel.max() <= 1e-13, "L={} form={} T={!r} m={} rel={:.3g}".format(L, form, T[worst[0]], worst[1],
                                                                                  rel.max())
