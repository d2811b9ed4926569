"""CPU oracle for contracted ERIs -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the C-ABI library and
its Python binding) never imports, links or executes anything here.

The arithmetic lives in ``eri_oracle.c`` (plain C, built twice: ``double`` and
``long double``); this module compiles it with gcc and marshals numpy arrays
through ctypes.  See the C file's header for what is computed and which
readings of the FusionRCG paper (Sec. II-A, Eqs. 1-3, 8, 17) it takes.

Parity status of each function (what pins it; the pins live in ``tests/``):
  boys       -- pinned: F_m(0), erf closed form, large-T asymptote, quadrature
                of the defining integral (mpmath).
  cart2sph   -- pinned: textbook l <= 2 solid harmonics, orthonormality under
                the Cartesian overlap metric, scipy spherical harmonics.
  eri        -- pinned: (ss|ss) closed form, brute-force quadrature of Eq. 1
                for every s/p class and spot d, f and g classes through
                (gg|gg), 8-fold permutation symmetry,
                rotational and translational invariance, Schwarz inequality,
                long-double adjudication.
  full_tensor, jk
             -- pinned: on s-only bases every (ij|kl) and hence J and K are
                given by the electrostatics of Gaussian charge clouds (closed
                form, independent of this package); J, K symmetric for a
                symmetric density; Coulomb and exchange energies
                tr(D J) >= 0 and tr(D K) >= 0 for a positive semidefinite D.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eri_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBS = {}
_LOCK = threading.Lock()


def _lib_path(long_double: bool) -> str:
    return os.path.join(_BUILD, "liboracle_ld.so" if long_double else "liboracle.so")


def build(force: bool = False) -> None:
    """Compile the oracle (both precisions) with gcc into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    for ld in (False, True):
        out = _lib_path(ld)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", out + ".tmp", "-lm"]
        if ld:
            cmd.insert(1, "-DORACLE_LONG_DOUBLE")
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)


def _lib(long_double: bool = False):
    with _LOCK:
        if long_double not in _LIBS:
            build()
            lib = ctypes.CDLL(_lib_path(long_double))
            pre = "oracle_ld_" if long_double else "oracle_"
            f = getattr(lib, pre + "eri_batch")
            f.restype = ctypes.c_int
            f.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int] + [ctypes.c_void_p] * 4 + \
                [ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            g = getattr(lib, pre + "boys_d")
            g.restype = None
            g.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
            h = getattr(lib, pre + "cart2sph_d")
            h.restype = None
            h.argtypes = [ctypes.c_int, ctypes.c_void_p]
            _LIBS[long_double] = (lib, f, g, h)
        return _LIBS[long_double]


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def nsph(l: int) -> int:
    return 2 * l + 1


def boys(L: int, T: float, long_double: bool = False) -> np.ndarray:
    """F_0..F_L at T (series + downward recursion, or erf + upward for T > 50)."""
    out = np.zeros(L + 1)
    _lib(long_double)[2](int(L), float(T), out.ctypes.data)
    return out


def cart2sph(l: int, long_double: bool = False) -> np.ndarray:
    """T^(l) of Eq. 8 as a [2l+1, ncart(l)] matrix (rows m = -l..l)."""
    out = np.zeros((2 * l + 1) * ncart(l))
    _lib(long_double)[3](int(l), out.ctypes.data)
    return out.reshape(2 * l + 1, ncart(l))


def block_sizes(basis, quartets, cart: bool = False) -> np.ndarray:
    n = ncart if cart else nsph
    ls = basis.shell_l[np.asarray(quartets, dtype=np.int64)]
    sz = np.ones(ls.shape[0], dtype=np.int64)
    for k in range(4):
        sz *= np.vectorize(n)(ls[:, k]) if ls.shape[0] else 1
    return sz


def offsets(basis, quartets, cart: bool = False) -> np.ndarray:
    sz = block_sizes(basis, quartets, cart)
    off = np.zeros(sz.shape[0] + 1, dtype=np.int64)
    np.cumsum(sz, out=off[1:])
    return off


def eri(basis, quartets, cart: bool = False, nthreads: int = 1, long_double: bool = False):
    """Contracted (ab|cd) for every quartet row (shell indices, taken in the
    given order).  Returns (values, offsets): block q is
    values[offsets[q]:offsets[q+1]], row-major over (a, b, c, d) components."""
    q = np.ascontiguousarray(np.asarray(quartets, dtype=np.int32).reshape(-1, 4))
    off = offsets(basis, q, cart)
    out = np.zeros(int(off[-1]))
    sl = np.ascontiguousarray(basis.shell_l, dtype=np.int32)
    sk = np.ascontiguousarray(basis.shell_nprim, dtype=np.int32)
    sc = np.ascontiguousarray(basis.shell_center, dtype=np.int32)
    sp = np.ascontiguousarray(basis.shell_prim, dtype=np.int32)
    ce = np.ascontiguousarray(basis.centers, dtype=np.float64)
    ex = np.ascontiguousarray(basis.exps, dtype=np.float64)
    co = np.ascontiguousarray(basis.coefs, dtype=np.float64)
    rc = _lib(long_double)[1](sl.ctypes.data, sk.ctypes.data, sc.ctypes.data, sp.ctypes.data, sl.shape[0],
                              ce.ctypes.data, ex.ctypes.data, co.ctypes.data, q.ctypes.data, q.shape[0],
                              1 if cart else 0, off.ctypes.data, out.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError("oracle: invalid basis or quartet list")
    return out, off


def basis_function_offsets(basis, cart: bool = False) -> np.ndarray:
    """First basis function of each shell (shells in order), and the total:
    [nshell + 1]."""
    n = np.array([ncart(l) if cart else nsph(l) for l in basis.shell_l], dtype=np.int64)
    return np.concatenate([[0], np.cumsum(n)])


def full_tensor(basis, cart: bool = False, nthreads: int = 1) -> np.ndarray:
    """The full ERI tensor (ij|kl) over the basis functions, [nbf]*4, from
    every ordered shell quartet (no symmetry used).  Small bases only."""
    ns = int(basis.shell_l.shape[0])
    idx = np.indices((ns, ns, ns, ns)).reshape(4, -1).T.astype(np.int32)
    v, off = eri(basis, idx, cart=cart, nthreads=nthreads)
    bf = basis_function_offsets(basis, cart)
    nbf = int(bf[-1])
    out = np.zeros((nbf, nbf, nbf, nbf))
    for q, (a, b, c, d) in enumerate(idx.tolist()):
        blk = v[off[q]:off[q + 1]].reshape(bf[a + 1] - bf[a], bf[b + 1] - bf[b], bf[c + 1] - bf[c], bf[d + 1] - bf[d])
        out[bf[a]:bf[a + 1], bf[b]:bf[b + 1], bf[c]:bf[c + 1], bf[d]:bf[d + 1]] = blk
    return out


def jk(basis, density: np.ndarray, cart: bool = False, nthreads: int = 1):
    """Coulomb and exchange matrices of a density D (FusionRCG Alg. 2, the
    digestion of the integrals into the Fock build):
        J_ij = sum_kl (ij|kl) D_kl,     K_ij = sum_kl (ik|jl) D_kl,
    written out over the full tensor."""
    g = full_tensor(basis, cart=cart, nthreads=nthreads)
    D = np.asarray(density, dtype=np.float64)
    J = np.einsum("ijkl,kl->ij", g, D)
    K = np.einsum("ikjl,kl->ij", g, D)
    return J, K
