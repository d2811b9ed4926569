"""Brute-force numerical quadrature of the ERI definition (the paper's Eq. 1),
independent of the Obara-Saika recurrences, the Boys function and the
closed-form normalisation: a test-side pin for the oracle.

1/r12 = (2/sqrt(pi)) int_0^inf exp(-t^2 r12^2) dt turns Eq. 1 into a t-integral
of a product of three one-dimensional problems.  For fixed t each is a 2-D
integral of a polynomial times a Gaussian exp(-(x-mu)^T M (x-mu)), which a
tensor Gauss-Hermite rule integrates exactly after the Cholesky substitution
x = mu + L^-T z.  The t-integral is mapped to s in [0, 1) by
t = k s / (1 - s) and done by Gauss-Legendre, doubling the node count until
two successive results agree.
"""
from __future__ import annotations

import math

import numpy as np

_GH_X, _GH_W = np.polynomial.hermite.hermgauss(10)  # exact to degree 19


def cart_tuples(l):
    return [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]


def norm_numeric(alpha: float, l: int) -> float:
    """1 / ||x^l exp(-alpha r^2)|| by Gauss-Hermite moments (no closed form)."""
    s = math.sqrt(2 * alpha)  # exp(-2 alpha x^2) = exp(-(s x)^2)
    m_x = np.sum(_GH_W * (_GH_X / s) ** (2 * l)) / s
    m_0 = np.sum(_GH_W) / s
    return 1.0 / math.sqrt(m_x * m_0 * m_0)


def _axis_factor(t, pa, pb, pc, pd, aa, ab, ac, ad, Ax, Bx, Cx, Dx):
    """I_x(t) for every t in the array: the 2-D integral over (x1, x2) of
    (x1-Ax)^pa (x1-Bx)^pb (x2-Cx)^pc (x2-Dx)^pd
    * exp(-aa(x1-Ax)^2 - ab(x1-Bx)^2 - ac(x2-Cx)^2 - ad(x2-Dx)^2 - t^2 (x1-x2)^2)."""
    t2 = t * t
    zeta, eta = aa + ab, ac + ad
    a11 = zeta + t2
    a22 = eta + t2
    a12 = -t2
    b1 = aa * Ax + ab * Bx
    b2 = ac * Cx + ad * Dx
    # det M and the constant of the completed square in cancellation-free
    # form: det = zeta eta + t^2 (zeta + eta); with P = b1/zeta, Q = b2/eta,
    # c0 - b^T M^-1 b = aa ab/zeta (A-B)^2 + ac ad/eta (C-D)^2
    #                   + t^2 zeta eta (P-Q)^2 / det
    det = zeta * eta + t2 * (zeta + eta)
    mu1 = (a22 * b1 - a12 * b2) / det
    mu2 = (a11 * b2 - a12 * b1) / det
    Px, Qx = b1 / zeta, b2 / eta
    const = aa * ab / zeta * (Ax - Bx) ** 2 + ac * ad / eta * (Cx - Dx) ** 2 + t2 * zeta * eta * (Px - Qx) ** 2 / det
    # Cholesky of M = [[a11, a12], [a12, a22]] = L L^T
    l11 = np.sqrt(a11)
    l21 = a12 / l11
    l22 = np.sqrt(det / a11)
    # x = mu + L^-T z ; L^-T = [[1/l11, -l21/(l11 l22)], [0, 1/l22]]
    z1 = _GH_X[:, None]
    z2 = _GH_X[None, :]
    w = _GH_W[:, None] * _GH_W[None, :]
    x1 = mu1[:, None, None] + (z1 / l11[:, None, None] - (l21 / (l11 * l22))[:, None, None] * z2)
    x2 = mu2[:, None, None] + z2 / l22[:, None, None]
    poly = (x1 - Ax) ** pa * (x1 - Bx) ** pb * (x2 - Cx) ** pc * (x2 - Dx) ** pd
    s = np.sum(w[None] * poly, axis=(1, 2))
    return np.exp(-const) * s / (l11 * l22)


def primitive_cart(ls, alphas, centers, nt):
    """Cartesian primitive integrals (unnormalised Gaussians) for every
    component combination, shape [nc_a, nc_b, nc_c, nc_d]."""
    aa, ab, ac, ad = alphas
    A, B, C, D = centers
    zeta, eta = aa + ab, ac + ad
    kappa = math.sqrt(zeta * eta / (zeta + eta))
    s, ws = np.polynomial.legendre.leggauss(nt)
    s = 0.5 * (s + 1.0)
    ws = 0.5 * ws
    t = kappa * s / (1.0 - s)
    dt = kappa * ws / (1.0 - s) ** 2
    tups = [cart_tuples(l) for l in ls]
    out = np.zeros([len(x) for x in tups])
    cache = {}
    for ia, ta in enumerate(tups[0]):
        for ib, tb in enumerate(tups[1]):
            for ic, tc in enumerate(tups[2]):
                for id_, td in enumerate(tups[3]):
                    prod = np.ones_like(t)
                    for k in range(3):
                        key = (k, ta[k], tb[k], tc[k], td[k])
                        if key not in cache:
                            cache[key] = _axis_factor(t, ta[k], tb[k], tc[k], td[k], aa, ab, ac, ad,
                                                      A[k], B[k], C[k], D[k])
                        prod = prod * cache[key]
                    out[ia, ib, ic, id_] = 2.0 / math.sqrt(math.pi) * np.sum(dt * prod)
    return out


def contracted_cart(basis, quartet, rtol=1e-13, nt0=64, nt_max=4096):
    """Contracted Cartesian (ab|cd) block by quadrature, each primitive
    normalised numerically like x^l exp(-a r^2)."""
    sh = [int(s) for s in quartet]
    ls = [int(basis.shell_l[s]) for s in sh]
    ctr = [basis.centers[basis.shell_center[s]] for s in sh]
    prims = []
    for s, l in zip(sh, ls):
        p0, k = int(basis.shell_prim[s]), int(basis.shell_nprim[s])
        prims.append([(basis.exps[p0 + i], basis.coefs[p0 + i] * norm_numeric(basis.exps[p0 + i], l))
                      for i in range(k)])

    def total(nt):
        acc = 0.0
        for (a, ca) in prims[0]:
            for (b, cb) in prims[1]:
                for (c, cc) in prims[2]:
                    for (d, cd) in prims[3]:
                        acc = acc + ca * cb * cc * cd * primitive_cart(ls, (a, b, c, d), ctr, nt)
        return acc

    nt = nt0
    prev = total(nt)
    while True:
        nt *= 2
        cur = total(nt)
        scale = np.max(np.abs(cur))
        if np.max(np.abs(cur - prev)) <= rtol * scale or nt >= nt_max:
            return cur
        prev = cur
