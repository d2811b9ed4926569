"""Reference blocks from the CPU oracle for the parity tests.

The oracle evaluates a quartet in whatever order it is given.  Its double
build is accurate to a tenth of the parity tolerance when the tighter shell
of each pair sits on the recurrence centre (pinned against the long-double
build in test_oracle_eri), so each quartet is evaluated in that orientation
and its block transposed back to the caller's order -- an exact permutation.
"""
import os

import numpy as np

import oracle

NS = [1, 3, 5, 7, 9]
NC = [1, 3, 6, 10, 15]


def tight_first(basis, q):
    q = np.array(q, dtype=np.int32).reshape(-1, 4)
    top = np.array([basis.exps[p:p + k].max() for p, k in zip(basis.shell_prim, basis.shell_nprim)])
    perm = np.tile(np.arange(4), (q.shape[0], 1))
    for j in (0, 2):
        sw = top[q[:, j]] < top[q[:, j + 1]]
        perm[sw, j], perm[sw, j + 1] = j + 1, j
    return np.take_along_axis(q, perm, axis=1), perm


def blocks(basis, quartets, cart=False, long_double=False, nthreads=None):
    """Oracle values for quartets in the caller's order (flat, with offsets)."""
    nthreads = nthreads or min(16, os.cpu_count() or 1)
    q = np.asarray(quartets, dtype=np.int32).reshape(-1, 4)
    qt, perm = tight_first(basis, q)
    v, off_t = oracle.eri(basis, qt, cart=cart, nthreads=nthreads, long_double=long_double)
    off = oracle.offsets(basis, q, cart)
    out = np.empty(int(off[-1]))
    n = NC if cart else NS
    for i in range(q.shape[0]):
        dims_t = [n[basis.shell_l[s]] for s in qt[i]]
        b = v[off_t[i]:off_t[i + 1]].reshape(dims_t)
        # qt[i][k] = q[i][perm[i][k]]: axis k of b belongs to user position perm[k]
        b = np.transpose(b, np.argsort(perm[i]))
        out[off[i]:off[i + 1]] = b.ravel()
    return out, off


def adjudicated(got, basis, quartets, cart=False, nthreads=None):
    """Reference for ``got``: the double oracle, with every quartet that has
    an element outside tolerance recomputed by the long-double build (the
    double build itself can miss the tolerance where HRR cancels digits)."""
    ref, off = blocks(basis, quartets, cart=cart, nthreads=nthreads)
    bad = ~within(got, ref)
    if bad.any():
        q = np.asarray(quartets, dtype=np.int32).reshape(-1, 4)
        qbad = np.unique(np.searchsorted(off, np.nonzero(bad)[0], side="right") - 1)
        ld, offl = blocks(basis, q[qbad], cart=cart, long_double=True, nthreads=nthreads)
        for k, qq in enumerate(qbad):
            ref[off[qq]:off[qq + 1]] = ld[offl[k]:offl[k + 1]]
    return ref, off


def within(got, ref, atol=1e-12, rtol=1e-10):
    """Elementwise parity criterion |got - ref| <= max(atol, rtol |ref|)."""
    return np.abs(got - ref) <= np.maximum(atol, rtol * np.abs(ref))


def report(got, ref):
    d = np.abs(got - ref)
    bad = ~within(got, ref)
    return "max|d| {:.3g}, max rel {:.3g}, {} of {} outside".format(
        d.max() if d.size else 0.0, (d / np.maximum(np.abs(ref), 1e-300)).max() if d.size else 0.0,
        int(bad.sum()), bad.size)
