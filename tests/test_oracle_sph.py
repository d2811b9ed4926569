"""Pins for the oracle's Cartesian-to-spherical coefficients T^(l) (the
paper's Eq. 8): textbook solid harmonics for l <= 3, orthonormality under the
Cartesian overlap metric, and agreement with scipy's spherical harmonics for
every l <= 4."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "solid_harmonics.txt")


def cart_tuples(l):
    return [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]


def dfact(n):
    return float(np.prod(np.arange(n, 0, -2))) if n > 0 else 1.0


def cart_overlap(l):
    """Overlap of the degree-l Cartesian components, each normalised like
    x^l exp(-a r^2): (i+i'-1)!!(j+j'-1)!!(k+k'-1)!! / (2l-1)!! when every sum
    is even, else 0 (separable Gaussian moments)."""
    ts = cart_tuples(l)
    S = np.zeros((len(ts), len(ts)))
    for p, a in enumerate(ts):
        for q, b in enumerate(ts):
            s = [a[k] + b[k] for k in range(3)]
            if all(x % 2 == 0 for x in s):
                S[p, q] = dfact(s[0] - 1) * dfact(s[1] - 1) * dfact(s[2] - 1) / dfact(2 * l - 1)
    return S


def test_textbook_values(oracle_mod):
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    ref = {l: np.zeros((2 * l + 1, (l + 1) * (l + 2) // 2)) for l in range(4)}
    for l, m, c, i, j, k in rows:
        l, m, i, j, k = int(l), int(m), int(i), int(j), int(k)
        ref[l][m + l, cart_tuples(l).index((i, j, k))] += float(c)
    for l in range(4):
        np.testing.assert_allclose(oracle_mod.cart2sph(l), ref[l], atol=1e-15, rtol=1e-15)


@pytest.mark.parametrize("l", range(5))
def test_orthonormal(oracle_mod, l):
    T = oracle_mod.cart2sph(l)
    np.testing.assert_allclose(T @ cart_overlap(l) @ T.T, np.eye(2 * l + 1), atol=2e-15)


@pytest.mark.parametrize("l", range(5))
def test_matches_scipy_harmonics(oracle_mod, l):
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(11 + l)
    pts = rng.normal(size=(40, 3))
    r = np.linalg.norm(pts, axis=1)
    theta = np.arccos(pts[:, 2] / r)
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    T = oracle_mod.cart2sph(l)
    mono = np.array([[x ** i * y ** j * z ** k for (i, j, k) in cart_tuples(l)] for x, y, z in pts])
    got = mono @ T.T  # [npt, 2l+1]
    for m in range(-l, l + 1):
        Y = sph_harm_y(l, abs(m), theta, phi)  # includes the Condon-Shortley phase
        if m > 0:
            yr = math.sqrt(2) * (-1) ** m * Y.real
        elif m < 0:
            yr = math.sqrt(2) * (-1) ** m * Y.imag
        else:
            yr = Y.real
        ref = math.sqrt(4 * math.pi / (2 * l + 1)) * r ** l * yr
        np.testing.assert_allclose(got[:, m + l], ref, rtol=1e-12, atol=1e-12)


def test_long_double_agrees(oracle_mod):
    for l in range(5):
        np.testing.assert_allclose(oracle_mod.cart2sph(l), oracle_mod.cart2sph(l, long_double=True), atol=1e-15)
