"""Pins for the oracle's Coulomb and exchange matrices (the digestion of
Alg. 2: J_ij = sum_kl (ij|kl) D_kl, K_ij = sum_kl (ik|jl) D_kl), each
independent of the oracle's own arithmetic:

* on an s-only basis every (ij|kl) is the electrostatic energy of two
  Gaussian charge clouds (closed form), so J and K follow by brute force;
* J and K are symmetric for a symmetric density;
* the Coulomb and exchange energies tr(D J) and tr(D K) are >= 0 for a
  positive semidefinite density (the ERI tensor is a positive kernel).
"""
import itertools
import math

import numpy as np
import pytest
from scipy.special import erf

from paper_2605_10312_gb300 import synth
from quad_eri import norm_numeric


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def _s_basis(n, seed):
    rng = np.random.default_rng(seed)
    bb = synth._BasisBuilder()
    for k in range(n):
        c = bb.add_center(rng.uniform(-2.0, 2.0, 3))
        bb.add_shell(0, c, [float(synth.log_uniform(rng, 0.1, 20.0, 1)[0])], [float(rng.uniform(0.3, 1.0))])
    return bb.build()


def _charge(a, c, X, i, j):
    """Total charge, exponent and centre of the product of s primitives i, j."""
    Ni, Nj = norm_numeric(a[i], 0), norm_numeric(a[j], 0)
    z = a[i] + a[j]
    P = (a[i] * X[i] + a[j] * X[j]) / z
    q = c[i] * c[j] * Ni * Nj * math.exp(-a[i] * a[j] / z * np.sum((X[i] - X[j]) ** 2)) * (math.pi / z) ** 1.5
    return q, z, P


def _gaussian_eri(basis, i, j, k, l):
    a, c, X = basis.exps, basis.coefs, basis.centers[basis.shell_center]
    q1, z, P = _charge(a, c, X, i, j)
    q2, e, Q = _charge(a, c, X, k, l)
    rho = z * e / (z + e)
    R = float(np.linalg.norm(P - Q))
    return q1 * q2 * (erf(math.sqrt(rho) * R) / R if R > 1e-8 else 2 * math.sqrt(rho / math.pi))


@pytest.mark.parametrize("seed", [1, 2])
def test_jk_s_basis_closed_form(oracle_mod, seed):
    n = 4
    basis = _s_basis(n, seed)
    rng = np.random.default_rng(seed + 10)
    D = rng.standard_normal((n, n))
    D = D + D.T
    g = np.zeros((n, n, n, n))
    for i, j, k, l in itertools.product(range(n), repeat=4):
        g[i, j, k, l] = _gaussian_eri(basis, i, j, k, l)
    Jref = np.zeros((n, n))
    Kref = np.zeros((n, n))
    for i, j, k, l in itertools.product(range(n), repeat=4):
        Jref[i, j] += g[i, j, k, l] * D[k, l]
        Kref[i, j] += g[i, k, j, l] * D[k, l]
    J, K = oracle_mod.jk(basis, D)
    assert np.allclose(J, Jref, rtol=1e-12, atol=1e-13)
    assert np.allclose(K, Kref, rtol=1e-12, atol=1e-13)


def test_jk_symmetry_and_energies(oracle_mod):
    basis, _ = synth.tiny_set()
    nbf = int(oracle_mod.basis_function_offsets(basis)[-1])
    rng = np.random.default_rng(4)
    C = rng.standard_normal((nbf, 3))
    D = C @ C.T  # positive semidefinite
    J, K = oracle_mod.jk(basis, D, nthreads=4)
    assert np.allclose(J, J.T, rtol=1e-12, atol=1e-13)
    assert np.allclose(K, K.T, rtol=1e-12, atol=1e-13)
    assert np.trace(D @ J) > 0
    assert np.trace(D @ K) > 0
    # the exchange energy of a rank-one density equals its Coulomb energy
    c = rng.standard_normal((nbf, 1))
    D1 = c @ c.T
    J1, K1 = oracle_mod.jk(basis, D1, nthreads=4)
    assert abs(np.trace(D1 @ J1) - np.trace(D1 @ K1)) <= 1e-12 * abs(np.trace(D1 @ J1))
