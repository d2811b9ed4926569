"""numpy interpreter for generator class programs (test-side only).

It evaluates a ``ClassProgram`` -- Phase-1 graph in its schedule order, then
the Phase-2 operation list -- for a batch of shell quartets given in the
program's orientation, so that the generator's graphs can be checked against
the oracle on the CPU before any kernel exists.  Pair quantities use their
textbook definitions and the Boys function comes from scipy's regularised
incomplete gamma function: nothing here is shared with the oracle or with the
device code.
"""
import math

import numpy as np
from scipy.special import gamma, gammainc

from quad_eri import norm_numeric


def boys_scipy(L, T):
    T = np.asarray(T, dtype=np.float64)
    out = np.empty(T.shape + (L + 1,))
    small = T < 1e-13
    Ts = np.where(small, 1.0, T)
    for m in range(L + 1):
        a = m + 0.5
        v = gamma(a) * gammainc(a, Ts) / (2.0 * Ts ** a)
        out[..., m] = np.where(small, 1.0 / (2 * m + 1) - T / (2 * m + 3), v)
    return out


def evaluate(prog, basis, quartets):
    """quartets: [nq, 4] shell indices already in the program's orientation
    (shells of angular momentum la, lb, lc, ld).  Returns [nq, nout]."""
    la, lb, lc, ld = prog.ls
    g, p2 = prog.g, prog.p2
    q = np.asarray(quartets)
    nq = q.shape[0]
    ctr = [basis.centers[basis.shell_center[q[:, k]]] for k in range(4)]
    H = np.zeros((prog.nh, nq))
    L = prog.L
    kmax = [int(basis.shell_nprim[q[:, k]].max()) for k in range(4)]
    for ia in range(kmax[0]):
        for ib in range(kmax[1]):
            for ic in range(kmax[2]):
                for id_ in range(kmax[3]):
                    idx = [ia, ib, ic, id_]
                    ok = np.ones(nq, dtype=bool)
                    al, co = [], []
                    for k, l in enumerate((la, lb, lc, ld)):
                        K = basis.shell_nprim[q[:, k]]
                        ok &= idx[k] < K
                        p = basis.shell_prim[q[:, k]] + np.minimum(idx[k], K - 1)
                        a = basis.exps[p]
                        al.append(a)
                        co.append(basis.coefs[p] * np.array([norm_numeric(x, l) for x in a]))
                    za, zb, zc, zd = al
                    zeta, eta = za + zb, zc + zd
                    P = (za[:, None] * ctr[0] + zb[:, None] * ctr[1]) / zeta[:, None]
                    Q = (zc[:, None] * ctr[2] + zd[:, None] * ctr[3]) / eta[:, None]
                    W = (zeta[:, None] * P + eta[:, None] * Q) / (zeta + eta)[:, None]
                    rho = zeta * eta / (zeta + eta)
                    T = rho * np.sum((P - Q) ** 2, axis=1)
                    kab = np.exp(-za * zb / zeta * np.sum((ctr[0] - ctr[1]) ** 2, axis=1))
                    kcd = np.exp(-zc * zd / eta * np.sum((ctr[2] - ctr[3]) ** 2, axis=1))
                    pref = 2 * math.pi ** 2.5 / (zeta * eta * np.sqrt(zeta + eta)) * kab * kcd
                    pref = pref * co[0] * co[1] * co[2] * co[3] * ok
                    F = boys_scipy(L, T) * pref[:, None]
                    coef = {}
                    for i in range(3):
                        coef[("PA", i)] = P[:, i] - ctr[0][:, i]
                        coef[("WP", i)] = W[:, i] - P[:, i]
                        coef[("QC", i)] = Q[:, i] - ctr[2][:, i]
                        coef[("WQ", i)] = W[:, i] - Q[:, i]
                    for k in range(1, 2 * L + 2):
                        coef[("c1z", k)] = k / (2 * zeta)
                        coef[("c2z", k)] = -k * rho / (2 * zeta * zeta)
                        coef[("c1e", k)] = k / (2 * eta)
                        coef[("c2e", k)] = -k * rho / (2 * eta * eta)
                        coef[("c3", k)] = k / (2 * (zeta + eta))
                    vals = [None] * len(g)
                    for v in prog.order:
                        ts = g.terms[v]
                        if not ts:
                            vals[v] = F[:, g.keys[v][2]]
                        else:
                            acc = 0.0
                            for c, p in ts:
                                acc = acc + coef[c] * vals[p]
                            vals[v] = acc
                    for v, t in g.target.items():
                        H[t] += vals[v]
    AB = ctr[0] - ctr[1]
    CD = ctr[2] - ctr[3]
    V = [None] * p2.nvals
    for i in range(prog.nh):
        V[i] = H[i]
    X = {"AB": AB, "CD": CD}
    for op in p2.ops:
        if op[0] == "hrr":
            _, d, hi, (sym, i), lo = op
            V[d] = V[hi] + X[sym][:, i] * V[lo]
        else:
            _, d, terms = op
            acc = 0.0
            for c, s in terms:
                acc = acc + c * V[s]
            V[d] = acc
    return np.stack([V[o] for o in p2.outputs], axis=1)


def run_encoded(enc, prog, basis, quartets):
    """Walk the encoded descriptors (the executor kernel's semantics) with
    the same per-primitive inputs as ``evaluate``; returns [nq, nout]."""
    from paper_2605_10312_gb300.gen.encode import coef_table
    la, lb, lc, ld = prog.ls
    q = np.asarray(quartets)
    nq = q.shape[0]
    ctr = [basis.centers[basis.shell_center[q[:, k]]] for k in range(4)]
    S = np.zeros((enc.nslot, nq))
    L = prog.L
    kmax = [int(basis.shell_nprim[q[:, k]].max()) for k in range(4)]
    for ia in range(kmax[0]):
        for ib in range(kmax[1]):
            for ic in range(kmax[2]):
                for id_ in range(kmax[3]):
                    idx = [ia, ib, ic, id_]
                    ok = np.ones(nq, dtype=bool)
                    al, co = [], []
                    for k, l in enumerate((la, lb, lc, ld)):
                        K = basis.shell_nprim[q[:, k]]
                        ok &= idx[k] < K
                        p = basis.shell_prim[q[:, k]] + np.minimum(idx[k], K - 1)
                        a = basis.exps[p]
                        al.append(a)
                        co.append(basis.coefs[p] * np.array([norm_numeric(x, l) for x in a]))
                    za, zb, zc, zd = al
                    zeta, eta = za + zb, zc + zd
                    P = (za[:, None] * ctr[0] + zb[:, None] * ctr[1]) / zeta[:, None]
                    Q = (zc[:, None] * ctr[2] + zd[:, None] * ctr[3]) / eta[:, None]
                    W = (zeta[:, None] * P + eta[:, None] * Q) / (zeta + eta)[:, None]
                    rho = zeta * eta / (zeta + eta)
                    T = rho * np.sum((P - Q) ** 2, axis=1)
                    kab = np.exp(-za * zb / zeta * np.sum((ctr[0] - ctr[1]) ** 2, axis=1))
                    kcd = np.exp(-zc * zd / eta * np.sum((ctr[2] - ctr[3]) ** 2, axis=1))
                    pref = 2 * math.pi ** 2.5 / (zeta * eta * np.sqrt(zeta + eta)) * kab * kcd
                    pref = pref * co[0] * co[1] * co[2] * co[3] * ok
                    F = boys_scipy(L, T) * pref[:, None]
                    geo = [[P[:, i] - ctr[0][:, i] for i in range(3)], [W[:, i] - P[:, i] for i in range(3)],
                           [Q[:, i] - ctr[2][:, i] for i in range(3)], [W[:, i] - Q[:, i] for i in range(3)]]
                    c1 = [1 / (2 * zeta), 1 / (2 * eta)]
                    c2 = [-rho / (2 * zeta * zeta), -rho / (2 * eta * eta)]
                    c3 = 1 / (2 * (zeta + eta))
                    for w0, w1, w2, w3 in enc.ph1.tolist():
                        dst, h = w0 & 0xFFFF, w0 >> 16
                        side, axis, k, k3 = (w3 >> 16) & 3, (w3 >> 18) & 3, (w3 >> 20) & 31, (w3 >> 25) & 31
                        if side == 2:
                            x = F[:, k]
                        else:
                            x = geo[2 * side][axis] * S[w1 & 0xFFFF] + geo[2 * side + 1][axis] * S[w1 >> 16]
                            if k:
                                x = x + k * c1[side] * S[w2 & 0xFFFF] + k * c2[side] * S[w2 >> 16]
                            if k3:
                                x = x + k3 * c3 * S[w3 & 0xFFFF]
                        if (w3 >> 30) & 1:
                            S[dst] = x
                        if h:
                            S[h - 1] += x
    ctab = coef_table()
    X = [ctr[0][:, i] - ctr[1][:, i] for i in range(3)] + [ctr[2][:, i] - ctr[3][:, i] for i in range(3)]
    out = np.zeros((nq, int(np.prod(enc.out_dims))))
    for w0, w1, w2, w3 in enc.ph2.tolist():
        kind = w0 & 3
        dst = w0 >> 16
        if kind == 0:
            S[dst] = S[w1 & 0xFFFF] + X[w2] * S[w1 >> 16]
        elif kind == 1:
            n = (w0 >> 2) & 7
            acc = S[dst].copy() if (w0 >> 5) & 1 else 0.0
            ss = [w1 & 0xFFFF, w1 >> 16, w2 & 0xFFFF, w2 >> 16]
            cc = [w3 & 255, (w3 >> 8) & 255, (w3 >> 16) & 255, w3 >> 24]
            for j in range(n):
                acc = acc + ctab[cc[j]] * S[ss[j]]
            S[dst] = acc
        else:
            out[:, w1] = S[dst]
    return out


def run_coop(cp, prog, basis, quartets):
    """Walk a team-cooperative program wave by wave (the coop executor's
    semantics, including slot reuse across waves); returns [nq, nout]."""
    from paper_2605_10312_gb300.gen.encode import coef_table
    la, lb, lc, ld = prog.ls
    q = np.asarray(quartets)
    nq = q.shape[0]
    ctr = [basis.centers[basis.shell_center[q[:, k]]] for k in range(4)]
    nh = cp.nh
    S = np.zeros((nh + cp.nslot, nq))   # ids < nh: H, else value slots
    L = prog.L
    kmax = [int(basis.shell_nprim[q[:, k]].max()) for k in range(4)]

    ILP = cp.ilp

    def waves(rows, steps):
        i = 0
        for st in steps:
            n = int(st) * cp.T * ILP
            yield rows[i:i + n]
            i += n

    for ia in range(kmax[0]):
        for ib in range(kmax[1]):
            for ic in range(kmax[2]):
                for id_ in range(kmax[3]):
                    idx = [ia, ib, ic, id_]
                    ok = np.ones(nq, dtype=bool)
                    al, co = [], []
                    for k, l in enumerate((la, lb, lc, ld)):
                        K = basis.shell_nprim[q[:, k]]
                        ok &= idx[k] < K
                        p = basis.shell_prim[q[:, k]] + np.minimum(idx[k], K - 1)
                        a = basis.exps[p]
                        al.append(a)
                        co.append(basis.coefs[p] * np.array([norm_numeric(x, l) for x in a]))
                    za, zb, zc, zd = al
                    zeta, eta = za + zb, zc + zd
                    P = (za[:, None] * ctr[0] + zb[:, None] * ctr[1]) / zeta[:, None]
                    Q = (zc[:, None] * ctr[2] + zd[:, None] * ctr[3]) / eta[:, None]
                    W = (zeta[:, None] * P + eta[:, None] * Q) / (zeta + eta)[:, None]
                    rho = zeta * eta / (zeta + eta)
                    T = rho * np.sum((P - Q) ** 2, axis=1)
                    kab = np.exp(-za * zb / zeta * np.sum((ctr[0] - ctr[1]) ** 2, axis=1))
                    kcd = np.exp(-zc * zd / eta * np.sum((ctr[2] - ctr[3]) ** 2, axis=1))
                    pref = 2 * math.pi ** 2.5 / (zeta * eta * np.sqrt(zeta + eta)) * kab * kcd
                    pref = pref * co[0] * co[1] * co[2] * co[3] * ok
                    F = boys_scipy(L, T) * pref[:, None]
                    geo = [[P[:, i] - ctr[0][:, i] for i in range(3)], [W[:, i] - P[:, i] for i in range(3)],
                           [Q[:, i] - ctr[2][:, i] for i in range(3)], [W[:, i] - Q[:, i] for i in range(3)]]
                    c1 = [1 / (2 * zeta), 1 / (2 * eta)]
                    c2 = [-rho / (2 * zeta * zeta), -rho / (2 * eta * eta)]
                    c3 = 1 / (2 * (zeta + eta))
                    for wave in waves(cp.ph1, cp.steps1):
                        res = []  # all lanes read before any writes (wave barrier semantics)
                        for w0, w1, w2, w3 in wave.tolist():
                            meta = w3 >> 16
                            if meta & 0x8000:
                                continue
                            dst, h = w0 & 0xFFFF, w0 >> 16
                            V = lambda s_: S[nh + s_]
                            if meta & 0x4000:
                                x = F[:, (meta >> 4) & 31]
                            else:
                                cgo, k, k3, side = meta & 15, (meta >> 4) & 31, (meta >> 9) & 15, (meta >> 13) & 1
                                axis = cgo - 6 * side
                                x = geo[2 * side][axis] * V(w1 & 0xFFFF) + geo[2 * side + 1][axis] * V(w1 >> 16)
                                if k:
                                    x = x + k * c1[side] * V(w2 & 0xFFFF) + k * c2[side] * V(w2 >> 16)
                                if k3:
                                    x = x + k3 * c3 * V(w3 & 0xFFFF)
                            res.append((dst, h, x))
                        for dst, h, x in res:
                            if dst != 0xFFFF:
                                S[nh + dst] = x
                            if h:
                                S[h - 1] += x
    ctab = coef_table()
    X = [ctr[0][:, i] - ctr[1][:, i] for i in range(3)] + [ctr[2][:, i] - ctr[3][:, i] for i in range(3)]
    out = np.full((nq, int(np.prod(cp.out_dims))), np.nan)
    for wave in waves(cp.ph2, cp.steps2):
        res = []
        for w0, w1, w2, w3 in wave.tolist():
            kind = w0 & 3
            dst = w0 >> 16
            if kind == 0:
                res.append(("v", dst, S[w1 & 0xFFFF] + X[w2] * S[w1 >> 16]))
            elif kind == 1:
                n = (w0 >> 2) & 7
                ss = [w1 & 0xFFFF, w1 >> 16, w2 & 0xFFFF, w2 >> 16]
                cc = [w3 & 255, (w3 >> 8) & 255, (w3 >> 16) & 255, w3 >> 24]
                acc = 0.0
                for j in range(n):
                    acc = acc + ctab[cc[j]] * S[ss[j]]
                res.append(("v", dst, acc))
            elif kind == 2:
                res.append(("o", w1, S[dst].copy()))
        for kind, a, x in res:
            if kind == "v":
                S[a] = x
            else:
                out[:, a] = x
    return out
