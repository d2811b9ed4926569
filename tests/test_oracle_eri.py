"""Pins for the oracle's contracted ERIs (the paper's Eq. 1 evaluated by
Eqs. 2, 3, 8, 17), each independent of the oracle's own arithmetic:

* (ss|ss) against the electrostatic energy of two Gaussian charge clouds;
* brute-force quadrature of Eq. 1 for every s/p class and spot d, f and g
  classes through (gg|gg);
* 8-fold permutational symmetry (each permutation runs different recurrences);
* rotational invariance through Wigner matrices built from scipy harmonics;
* translational invariance, the Schwarz inequality, sph == cart for l <= 1;
* the long-double build, to bound the rounding of the double build.
"""
import itertools
import math

import numpy as np
import pytest
from scipy.special import erf, sph_harm_y

from paper_2605_10312_gb300 import synth
from quad_eri import contracted_cart, norm_numeric

NS = [1, 3, 5, 7, 9]
NC = [1, 3, 6, 10, 15]


def _basis_for(ls, K, seed, box=3.0, exp_range=(0.1, 20.0)):
    return synth.class_sweep(ls, 1, kset=(K,), seed=seed, box_angstrom=box, exp_range=exp_range)


def test_ssss_gaussian_charges(oracle_mod):
    """For s functions the bra product is a spherical Gaussian charge of total
    q = <ab> centred at P with exponent zeta; two such clouds interact as
    q1 q2 erf(sqrt(rho) R) / R, rho = zeta eta / (zeta + eta)."""
    rng = np.random.default_rng(3)
    for trial in range(40):
        basis, q = synth.class_sweep((0, 0, 0, 0), 1, kset=(1,), seed=100 + trial, box_angstrom=4.0,
                                     exp_range=(0.05, 500.0))
        v, _ = oracle_mod.eri(basis, q)
        a = basis.exps[:4]
        c = basis.coefs[:4]
        X = basis.centers[:4]
        N = [norm_numeric(x, 0) for x in a]
        zeta, eta = a[0] + a[1], a[2] + a[3]
        P = (a[0] * X[0] + a[1] * X[1]) / zeta
        Q = (a[2] * X[2] + a[3] * X[3]) / eta
        q1 = c[0] * c[1] * N[0] * N[1] * math.exp(-a[0] * a[1] / zeta * np.sum((X[0] - X[1]) ** 2)) * (math.pi / zeta) ** 1.5
        q2 = c[2] * c[3] * N[2] * N[3] * math.exp(-a[2] * a[3] / eta * np.sum((X[2] - X[3]) ** 2)) * (math.pi / eta) ** 1.5
        rho = zeta * eta / (zeta + eta)
        R = float(np.linalg.norm(P - Q))
        ref = q1 * q2 * (erf(math.sqrt(rho) * R) / R if R > 1e-8 else 2 * math.sqrt(rho / math.pi))
        assert abs(v[0] - ref) <= 1e-13 * abs(ref) + 1e-300, (trial, v[0], ref)


SP_CLASSES = [c for c in itertools.product((0, 1), repeat=4)]
D_CLASSES = [(2, 0, 0, 0), (0, 2, 0, 0), (2, 2, 0, 0), (2, 0, 1, 0), (1, 1, 2, 0), (0, 0, 0, 2), (2, 1, 1, 2)]
# f and g shells: Obara-Saika terms with k = 2, 3 (and cross terms of k3 up
# to 4) first appear here; the Gauss-Hermite rule stays exact through l = 4
FG_CLASSES = [(3, 0, 0, 0), (0, 3, 0, 0), (4, 0, 0, 0), (0, 0, 0, 4), (3, 1, 0, 0), (3, 0, 2, 0), (4, 0, 1, 0),
              (3, 3, 0, 0), (4, 1, 3, 0), (4, 4, 4, 0), (3, 3, 3, 3), (4, 4, 4, 4)]


@pytest.mark.parametrize("ls", SP_CLASSES + D_CLASSES + FG_CLASSES)
def test_quadrature(oracle_mod, ls):
    K = 2 if sum(ls) <= 4 else 1
    basis, q = _basis_for(ls, K, seed=500 + 7 * sum(l * 5 ** i for i, l in enumerate(ls)))
    ref = contracted_cart(basis, q[0]).ravel()
    v, _ = oracle_mod.eri(basis, q, cart=True)
    scale = np.max(np.abs(ref))
    assert np.all(np.abs(v - ref) <= 1e-10 * np.abs(ref) + 1e-11 * scale), np.max(np.abs(v - ref)) / scale


PERMS = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2), (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]


@pytest.mark.parametrize("ls", [(1, 0, 2, 1), (2, 1, 0, 3), (3, 3, 1, 2), (4, 2, 3, 1), (4, 4, 4, 4)])
def test_permutation_symmetry(oracle_mod, ls):
    n = 1 if sum(ls) >= 14 else 4
    basis, q = synth.class_sweep(ls, n, kset=(1, 2), seed=77 + sum(ls), box_angstrom=3.0, exp_range=(0.1, 30.0))
    for qi in range(n):
        blocks = {}
        for p in PERMS:
            # long double: the double build loses digits to HRR cancellation
            # when the diffuse shell of a pair sits on the recurrence centre
            v, _ = oracle_mod.eri(basis, q[qi][list(p)][None], long_double=True)
            blocks[p] = v.reshape([NS[ls[i]] for i in p])
        ref = blocks[PERMS[0]]
        scale = np.max(np.abs(ref))
        for p in PERMS[1:]:
            inv = np.argsort(p)
            got = np.transpose(blocks[p], inv)
            # HRR with |A-B| of several bohr cancels digits (about six in
            # the worst orientation here), so the floor is absolute: 1/10 of
            # the 1e-12 parity tolerance
            assert np.all(np.abs(got - ref) <= 1e-13 + 1e-12 * np.abs(ref)), (p, np.max(np.abs(got - ref)))


def _real_solid(l, pts):
    r = np.linalg.norm(pts, axis=1)
    th = np.arccos(np.clip(pts[:, 2] / r, -1, 1))
    ph = np.arctan2(pts[:, 1], pts[:, 0])
    out = np.zeros((pts.shape[0], 2 * l + 1))
    for m in range(-l, l + 1):
        Y = sph_harm_y(l, abs(m), th, ph)
        yr = math.sqrt(2) * (-1) ** m * (Y.real if m > 0 else Y.imag) if m != 0 else Y.real
        out[:, m + l] = math.sqrt(4 * math.pi / (2 * l + 1)) * r ** l * yr
    return out


def _wigner_real(l, R, rng):
    """D with S_l(R u) = D S_l(u), by least squares over random points."""
    u = rng.normal(size=(60, 3))
    A = _real_solid(l, u)
    Bm = _real_solid(l, u @ R.T)
    DT, *_ = np.linalg.lstsq(A, Bm, rcond=None)
    return DT.T


@pytest.mark.parametrize("ls", [(1, 1, 1, 1), (2, 1, 2, 0), (3, 2, 1, 1), (2, 2, 2, 2), (4, 3, 2, 1)])
def test_rotational_invariance(oracle_mod, ls):
    rng = np.random.default_rng(900 + sum(ls))
    basis, q = synth.class_sweep(ls, 2, kset=(1, 2), seed=31 + sum(ls), box_angstrom=3.0, exp_range=(0.1, 30.0))
    R = synth.random_rotation(rng)
    rot = synth.with_centers(basis, basis.centers @ R.T)
    v0, off = oracle_mod.eri(basis, q, long_double=True)
    v1, _ = oracle_mod.eri(rot, q, long_double=True)
    D = [_wigner_real(l, R, rng) for l in ls]
    shape = [NS[l] for l in ls]
    for k in range(q.shape[0]):
        b0 = v0[off[k]:off[k + 1]].reshape(shape)
        b1 = v1[off[k]:off[k + 1]].reshape(shape)
        pred = np.einsum("ai,bj,ck,dl,ijkl->abcd", D[0], D[1], D[2], D[3], b0)
        scale = np.max(np.abs(b0))
        assert np.max(np.abs(pred - b1)) <= 1e-11 * scale
        assert abs(np.linalg.norm(b0) - np.linalg.norm(b1)) <= 1e-12 * np.linalg.norm(b0)


def test_translational_invariance(oracle_mod):
    basis, q = synth.class_sweep((3, 1, 2, 2), 3, kset=(1, 3), seed=41, box_angstrom=3.0)
    shifted = synth.with_centers(basis, basis.centers + np.array([3.7, -12.1, 5.5]))
    q = _tight_first(basis, q)
    v0, _ = oracle_mod.eri(basis, q)
    v1, _ = oracle_mod.eri(shifted, q)
    assert np.all(np.abs(v0 - v1) <= 1e-14 + 1e-12 * np.abs(v0))


def test_schwarz_inequality(oracle_mod):
    for ls in [(1, 0, 1, 1), (2, 1, 2, 2), (3, 3, 2, 0)]:
        basis, q = synth.class_sweep(ls, 4, kset=(1, 2), seed=55 + sum(ls), box_angstrom=4.0)
        for qi in range(q.shape[0]):
            a, b, c, d = q[qi]
            abcd, _ = oracle_mod.eri(basis, q[qi][None])
            abab, _ = oracle_mod.eri(basis, np.array([[a, b, a, b]]))
            cdcd, _ = oracle_mod.eri(basis, np.array([[c, d, c, d]]))
            na, nb, nc, nd = (NS[x] for x in ls)
            abcd = abcd.reshape(na * nb, nc * nd)
            dab = np.diag(abab.reshape(na * nb, na * nb))
            dcd = np.diag(cdcd.reshape(nc * nd, nc * nd))
            assert np.all(dab > 0) and np.all(dcd > 0)
            bound = np.sqrt(dab)[:, None] * np.sqrt(dcd)[None, :]
            assert np.all(np.abs(abcd) <= bound * (1 + 1e-12))


@pytest.mark.parametrize("ls", [(1, 0, 0, 0), (1, 1, 1, 1), (0, 1, 1, 0)])
def test_sph_equals_cart_for_sp(oracle_mod, ls):
    # for l <= 1 the spherical functions are the Cartesian ones reordered (y, z, x)
    basis, q = synth.class_sweep(ls, 3, kset=(3,), seed=61)
    vs, off = oracle_mod.eri(basis, q)
    vc, _ = oracle_mod.eri(basis, q, cart=True)
    perm = {0: [0], 1: [1, 2, 0]}
    for k in range(q.shape[0]):
        bc = vc[off[k]:off[k + 1]].reshape([NC[l] for l in ls])
        for i, l in enumerate(ls):
            bc = np.take(bc, perm[l], axis=i)
        np.testing.assert_array_equal(vs[off[k]:off[k + 1]], bc.ravel())


def _tight_first(basis, q):
    """Each pair ordered so that the shell holding the largest exponent comes
    first (it is the centre the recurrences build on)."""
    q = q.copy()
    top = np.array([basis.exps[p:p + k].max() for p, k in zip(basis.shell_prim, basis.shell_nprim)])
    for i in range(q.shape[0]):
        for j in (0, 2):
            if top[q[i, j]] < top[q[i, j + 1]]:
                q[i, j], q[i, j + 1] = q[i, j + 1], q[i, j]
    return q


@pytest.mark.parametrize("ls", [(2, 2, 1, 1), (3, 3, 3, 3), (4, 4, 4, 4), (4, 0, 4, 0), (1, 4, 2, 3)])
@pytest.mark.parametrize("box", [3.0, 10.0])
def test_long_double_adjudication(oracle_mod, ls, box):
    """With the tighter shell of each pair on the recurrence centre, the double
    build stays within 1/10 of the parity tolerance (1e-12 absolute, 1e-10
    relative) of the long-double build, on compact and sparse geometries."""
    n = 2 if sum(ls) >= 12 else 12
    basis, q = synth.class_sweep(ls, n, kset=(1, 2), seed=2000 + sum(ls), box_angstrom=box)
    q = _tight_first(basis, q)
    v, _ = oracle_mod.eri(basis, q)
    w, _ = oracle_mod.eri(basis, q, long_double=True)
    assert np.all(np.abs(v - w) <= np.maximum(1e-12, 1e-10 * np.abs(w)) * 0.1)
