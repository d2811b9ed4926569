"""Pins for the oracle's Boys function F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt
(the base values of the paper's Phase 1, Sec. II-A): special values, the erf
closed form of F_0, the large-T asymptote, and high-precision quadrature of
the defining integral."""
import math

import numpy as np
import pytest
from scipy.special import erf


def test_boys_at_zero(oracle_mod):
    # F_m(0) = 1 / (2m + 1)
    F = oracle_mod.boys(16, 0.0)
    np.testing.assert_allclose(F, 1.0 / (2 * np.arange(17) + 1), rtol=1e-15, atol=0)


@pytest.mark.parametrize("T", [1e-8, 0.3, 1.0, 7.5, 29.0, 49.9, 50.1, 80.0, 700.0, 3.0e5])
def test_boys_f0_erf(oracle_mod, T):
    # F_0(T) = (1/2) sqrt(pi/T) erf(sqrt(T))
    ref = 0.5 * math.sqrt(math.pi / T) * erf(math.sqrt(T))
    assert abs(oracle_mod.boys(0, T)[0] - ref) <= 2e-15 * ref


@pytest.mark.parametrize("T", [200.0, 1.0e3, 3.0e5])
def test_boys_asymptote(oracle_mod, T):
    # F_m(T) -> (2m-1)!! / 2^(m+1) * sqrt(pi / T^(2m+1)) for T >> m
    F = oracle_mod.boys(16, T)
    for m in range(17):
        dfm = float(np.prod(np.arange(2 * m - 1, 0, -2))) if m > 0 else 1.0
        ref = dfm / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
        assert abs(F[m] - ref) <= 1e-14 * ref


def _boys_mp(m, T, mp):
    """High-precision F_m(T) by adaptive quadrature of the defining integral.
    For T <= 100 the integral over t in [0, 1] is taken as it stands; for
    larger T, where exp(-T t^2) is sharply peaked, it is written in
    s = t sqrt(T) as T^-(m+1/2) int_0^sqrt(T) s^(2m) exp(-s^2) ds and split at
    s = 1/4, 1/2, 1, 2, ... 64.  Cross-checked against the lower incomplete
    gamma form gamma(m+1/2, T) / (2 T^(m+1/2))."""
    if T == 0:
        return mp.mpf(1) / (2 * m + 1)
    if T <= 100:
        q = mp.quad(lambda t: t ** (2 * m) * mp.exp(-T * t * t), [0, 1], maxdegree=12)
    else:
        rt = mp.sqrt(T)
        f = lambda s: s ** (2 * m) * mp.exp(-s * s)
        pts = [mp.mpf(0)] + [mp.mpf(2) ** k for k in range(-2, 7) if mp.mpf(2) ** k < rt] + [rt]
        q = mp.quad(f, pts, maxdegree=12) / rt ** (2 * m + 1)
    g = mp.gammainc(m + mp.mpf(1) / 2, 0, T) / (2 * T ** (m + mp.mpf(1) / 2))
    assert abs(q - g) <= mp.mpf(10) ** -20 * abs(g)
    return q


def test_boys_quadrature_200(oracle_mod):
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 34
    rng = np.random.default_rng(20260)
    # 200 seeded T spread over [0, 3e5]: log-uniform plus the series/recursion seam
    Ts = np.concatenate([np.exp(rng.uniform(math.log(1e-6), math.log(3e5), 190)),
                         np.array([0.0, 1e-12, 49.999, 50.0, 50.001, 12.0, 36.0, 100.0, 1e4, 3e5])])
    worst = 0.0
    for T in Ts:
        F = oracle_mod.boys(16, float(T))
        for m in range(17):
            ref = _boys_mp(m, mp.mpf(float(T)), mp)
            rel = abs(F[m] - float(ref)) / float(ref)
            worst = max(worst, rel)
    assert worst <= 1e-14, worst


def test_boys_long_double_agrees(oracle_mod):
    rng = np.random.default_rng(5)
    for T in np.exp(rng.uniform(-10, 12, 50)):
        a = oracle_mod.boys(16, float(T))
        b = oracle_mod.boys(16, float(T), long_double=True)
        np.testing.assert_allclose(a, b, rtol=1e-14, atol=0)
