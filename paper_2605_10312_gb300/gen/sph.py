"""Cartesian-to-spherical coefficients T^(l) (the paper's Eq. 8) for the CUDA
path, built from the recurrence of real solid harmonics (Helgaker, Jorgensen
and Olsen, Molecular Electronic-Structure Theory, Sec. 6.4.4):

  S_00 = 1
  S_{l+1, l+1}  = sqrt(2^d (2l+1)/(2l+2)) (x S_{ll} - (1-d) y S_{l,-l})
  S_{l+1,-l-1}  = sqrt(2^d (2l+1)/(2l+2)) (y S_{ll} + (1-d) x S_{l,-l})
  S_{l+1, m}    = ((2l+1) z S_{lm} - sqrt((l+m)(l-m)) r^2 S_{l-1,m})
                  / sqrt((l+m+1)(l-m+1)),    |m| <= l
with d = 1 if l = 0 else 0.  Racah normalisation: with every Cartesian
component of a shell normalised like x^l exp(-a r^2) the spherical functions
are normalised.  Rows m = -l..l, columns in Cartesian order.
"""
from functools import lru_cache
import math

import numpy as np

from . import cart


def _pmul(p, mono, c):
    out = {}
    for k, v in p.items():
        kk = (k[0] + mono[0], k[1] + mono[1], k[2] + mono[2])
        out[kk] = out.get(kk, 0.0) + c * v
    return out


def _padd(*ps):
    out = {}
    for p in ps:
        for k, v in p.items():
            out[k] = out.get(k, 0.0) + v
    return out


@lru_cache(maxsize=None)
def _solid(lmax: int):
    S = {0: {0: {(0, 0, 0): 1.0}}}
    for l in range(lmax):
        d = 1 if l == 0 else 0
        f = math.sqrt(2.0 ** d * (2 * l + 1) / (2 * l + 2))
        nxt = {}
        nxt[l + 1] = _padd(_pmul(S[l][l], (1, 0, 0), f), _pmul(S[l][-l], (0, 1, 0), -f * (1 - d)))
        nxt[-l - 1] = _padd(_pmul(S[l][l], (0, 1, 0), f), _pmul(S[l][-l], (1, 0, 0), f * (1 - d)))
        for m in range(-l, l + 1):
            a = _pmul(S[l][m], (0, 0, 1), 2 * l + 1)
            parts = [a]
            if abs(m) <= l - 1:
                c = -math.sqrt((l + m) * (l - m))
                pm = S[l - 1][m]
                parts += [_pmul(pm, (2, 0, 0), c), _pmul(pm, (0, 2, 0), c), _pmul(pm, (0, 0, 2), c)]
            den = math.sqrt((l + m + 1) * (l - m + 1))
            nxt[m] = {k: v / den for k, v in _padd(*parts).items()}
        S[l + 1] = nxt
    return S


@lru_cache(maxsize=None)
def matrix(l: int) -> np.ndarray:
    """T^(l) as a [2l+1, ncart(l)] array."""
    S = _solid(max(l, 1))[l]
    T = np.zeros((2 * l + 1, cart.ncart(l)))
    for m in range(-l, l + 1):
        for mono, c in S[m].items():
            if abs(c) > 1e-14:
                T[m + l, cart.index(mono)] += c
    T[np.abs(T) < 1e-14] = 0.0
    return T
