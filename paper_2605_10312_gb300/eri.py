"""Python binding of the C ABI in include/eri.h (argument marshalling only).

Every step of the integral path runs in the library's CUDA kernels; PyTorch
supplies device memory and streams.  Loading fails loudly when the library
has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

ERI_OK = 0
ERRORS = {-1: "EINVAL", -2: "EUNSUPPORTED", -3: "ENOMEM", -4: "ECUDA", -5: "EBUSY", -6: "ETIMEOUT", -7: "ESTATE"}
AXIS_RULES = {"prose": 0, "literal": 1, "common": 2}
SCHEDULES = {"dsa": 0, "level": 1}
SPH_MODES = {"stepwise": 0, "materialize": 1, "cart": 2}
TIERS = {"auto": 0, "reg": 1, "shared": 2, "global": 3, "coop": 4}
TIERS_INV = {0: "setup", 1: "reg", 2: "shared", 3: "global", 4: "coop", 5: "persistent"}
ORIENTATIONS = {"split": 0, "l": 1, "tight": 2}
VOTES = {"auto": 0, "off": 1, "on": 2}


class EriError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("{} ({}): {}".format(ERRORS.get(code, code), code, msg))
        self.code = code


class _Shell(ctypes.Structure):
    _fields_ = [("l", ctypes.c_int32), ("nprim", ctypes.c_int32), ("center", ctypes.c_int32),
                ("prim_offset", ctypes.c_int32)]


class _Basis(ctypes.Structure):
    _fields_ = [("centers", ctypes.c_void_p), ("ncenter", ctypes.c_int32), ("exponents", ctypes.c_void_p),
                ("coefs", ctypes.c_void_p), ("nprim_total", ctypes.c_int32)]


class _Opts(ctypes.Structure):
    _fields_ = [("axis_rule", ctypes.c_int32), ("schedule", ctypes.c_int32), ("sph_mode", ctypes.c_int32),
                ("tier", ctypes.c_int32), ("orientation", ctypes.c_int32), ("streams", ctypes.c_int32),
                ("digest", ctypes.c_int32), ("votes", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("ordered", ctypes.c_int32)]


_lib = None


def library(path: str = LIB):
    """The loaded liberi.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("CUDA library {} is not built; run __graft_entry__.build()".format(path))
        lib = ctypes.CDLL(path)
        lib.eri_plan.restype = ctypes.c_int
        lib.eri_plan.argtypes = [ctypes.POINTER(_Shell), ctypes.c_int32, ctypes.POINTER(_Basis), ctypes.c_void_p,
                                 ctypes.c_int64, ctypes.POINTER(_Opts), ctypes.POINTER(ctypes.c_void_p)]
        lib.eri_plan_mixed.restype = ctypes.c_int
        lib.eri_plan_mixed.argtypes = [ctypes.POINTER(_Shell), ctypes.c_int32, ctypes.POINTER(_Basis),
                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double,
                                       ctypes.POINTER(_Opts), ctypes.POINTER(ctypes.c_void_p)]
        lib.eri_plan_on_stream.restype = ctypes.c_int
        lib.eri_plan_on_stream.argtypes = [ctypes.POINTER(_Shell), ctypes.c_int32, ctypes.POINTER(_Basis),
                                           ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double,
                                           ctypes.POINTER(_Opts), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
        lib.eri_digest_jk.restype = ctypes.c_int
        lib.eri_digest_jk.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.eri_compute_jk.restype = ctypes.c_int
        lib.eri_compute_jk.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
        lib.eri_mol_create.restype = ctypes.c_int
        lib.eri_mol_create.argtypes = [ctypes.POINTER(_Shell), ctypes.c_int32, ctypes.POINTER(_Basis),
                                       ctypes.POINTER(_Opts), ctypes.POINTER(ctypes.c_void_p)]
        lib.eri_mol_destroy.restype = ctypes.c_int
        lib.eri_mol_destroy.argtypes = [ctypes.c_void_p]
        lib.eri_plan_on_mol.restype = ctypes.c_int
        lib.eri_plan_on_mol.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_double, ctypes.POINTER(_Opts), ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]
        lib.eri_plan_launch_precision.restype = ctypes.c_int
        lib.eri_plan_launch_precision.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.eri_output_count.restype = ctypes.c_int64
        lib.eri_output_count.argtypes = [ctypes.c_void_p]
        lib.eri_output_offsets.restype = ctypes.c_int
        lib.eri_output_offsets.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        lib.eri_compute.restype = ctypes.c_int
        lib.eri_compute.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.eri_compute_host.restype = ctypes.c_int
        lib.eri_compute_host.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.eri_plan_stats.restype = ctypes.c_int
        lib.eri_plan_stats.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.eri_plan_set_timing.restype = ctypes.c_int
        lib.eri_plan_set_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.eri_plan_launch_count.restype = ctypes.c_int
        lib.eri_plan_launch_count.argtypes = [ctypes.c_void_p]
        lib.eri_plan_launch_info.restype = ctypes.c_int
        lib.eri_plan_launch_info.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]
        lib.eri_compute_fixed_scratch.restype = ctypes.c_int
        lib.eri_compute_fixed_scratch.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.eri_schwarz.restype = ctypes.c_int
        lib.eri_schwarz.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.eri_set_class_tier.restype = ctypes.c_int
        lib.eri_set_class_tier.argtypes = [ctypes.c_int] * 5
        lib.eri_set_class_votes.restype = ctypes.c_int
        lib.eri_set_class_votes.argtypes = [ctypes.c_int] * 5
        lib.eri_plan_graph_capture.restype = ctypes.c_int
        lib.eri_plan_graph_capture.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.eri_plan_graph_capture_jk.restype = ctypes.c_int
        lib.eri_plan_graph_capture_jk.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_void_p]
        lib.eri_plan_graph_launch.restype = ctypes.c_int
        lib.eri_plan_graph_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        lib.eri_screen_quartets.restype = ctypes.c_int
        lib.eri_screen_quartets.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                            ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.c_void_p]
        lib.eri_class_shapes.restype = ctypes.c_int
        lib.eri_class_shapes.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p, ctypes.c_int]
        lib.eri_set_class_shape.restype = ctypes.c_int
        lib.eri_set_class_shape.argtypes = [ctypes.c_int] * 7
        lib.eri_plan_launch_shape.restype = ctypes.c_int
        lib.eri_plan_launch_shape.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        lib.eri_boys_eval.restype = ctypes.c_int
        lib.eri_boys_eval.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p]
        lib.eri_plan_destroy.restype = ctypes.c_int
        lib.eri_plan_destroy.argtypes = [ctypes.c_void_p]
        lib.eri_last_error.restype = ctypes.c_char_p
        lib.eri_last_error.argtypes = []
        _lib = lib
    return _lib


def _check(rc):
    if rc != ERI_OK:
        raise EriError(rc, library().eri_last_error().decode())


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _marshal_basis(basis):
    """(shell array, eri_basis struct, arrays to keep alive) for a Basis."""
    ns = int(basis.shell_l.shape[0])
    # eri_shell records {l, nprim, center, prim_offset}, int32 each
    shv = np.empty((max(ns, 1), 4), dtype=np.int32)
    if ns:
        shv[:, 0] = basis.shell_l
        shv[:, 1] = basis.shell_nprim
        shv[:, 2] = basis.shell_center
        shv[:, 3] = basis.shell_prim
    keep = [np.ascontiguousarray(basis.centers, dtype=np.float64), np.ascontiguousarray(basis.exps, dtype=np.float64),
            np.ascontiguousarray(basis.coefs, dtype=np.float64), shv]
    b = _Basis(keep[0].ctypes.data, int(keep[0].shape[0]), keep[1].ctypes.data, keep[2].ctypes.data,
               int(keep[1].shape[0]))
    return shv.ctypes.data_as(ctypes.POINTER(_Shell)), ns, b, keep


class Mol:
    """A molecule kept on the device (eri_mol_create): shells and the
    primitive-pair records of every shell pair, computed once."""

    def __init__(self, basis, orientation="split"):
        lib = library()
        sh, ns, b, keep = _marshal_basis(basis)
        o = _Opts(0, 0, 0, 0, ORIENTATIONS[orientation], 0, 0)
        h = ctypes.c_void_p()
        _check(lib.eri_mol_create(sh, ns, ctypes.byref(b), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.basis = basis
        self.orientation = orientation

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            library().eri_mol_destroy(self._h)
            self._h = None


class Plan:
    """A device-resident plan for one quartet list (see eri_plan)."""

    def __init__(self, basis, quartets, axis_rule="prose", schedule="dsa", sph_mode="stepwise", tier="auto",
                 orientation="split", qbound=None, fp32_below=None, streams=0, stream=None, digest=False,
                 mol=None, votes="auto", persistent=False, ordered=False):
        """qbound/fp32_below: mixed precision (eri_plan_mixed) -- quartets whose
        bound is below fp32_below run their recurrences in FP32.  stream: a
        stream-ordered plan (eri_plan_on_stream) whose device memory lives and
        dies on that stream; compute it on the same stream.  mol: a Mol whose
        shells the quartets index (eri_plan_on_mol); basis is then ignored.
        ordered: the parts of a multi-part quartet add into its block in a
        fixed order, one launch round each (bitwise reproducible); else they
        run together and reduce atomically (fewer launches)."""
        lib = library()
        q = np.ascontiguousarray(np.asarray(quartets, dtype=np.int32).reshape(-1, 4))
        if mol is not None:
            self._keep = [q]
        else:
            sh, ns, b, keep = _marshal_basis(basis)
            self._keep = keep + [q]
        o = _Opts(AXIS_RULES[axis_rule], SCHEDULES[schedule], SPH_MODES[sph_mode], TIERS[tier],
                  ORIENTATIONS[orientation], int(streams), 1 if digest else 0, VOTES[votes],
                  1 if persistent else 0, 1 if ordered else 0)
        h = ctypes.c_void_p()
        qb = None
        if qbound is not None:
            qb = np.ascontiguousarray(np.asarray(qbound, dtype=np.float64).reshape(-1))
            if qb.shape[0] != q.shape[0]:
                raise ValueError("qbound needs one entry per quartet")
        if mol is not None:
            if orientation != mol.orientation:
                raise ValueError("orientation differs from the molecule's")
            _check(lib.eri_plan_on_mol(mol._h, q.ctypes.data, q.shape[0], None if qb is None else qb.ctypes.data,
                                       float(fp32_below if fp32_below is not None else 0.0), ctypes.byref(o),
                                       None if stream is None else _stream_handle(stream), ctypes.byref(h)))
            self._mol = mol  # the plan must not outlive the molecule
        elif stream is not None:
            _check(lib.eri_plan_on_stream(sh, ns, ctypes.byref(b), q.ctypes.data, q.shape[0],
                                          None if qb is None else qb.ctypes.data,
                                          float(fp32_below if fp32_below is not None else 0.0), ctypes.byref(o),
                                          _stream_handle(stream), ctypes.byref(h)))
        elif qbound is None:
            _check(lib.eri_plan(sh, ns, ctypes.byref(b), q.ctypes.data, q.shape[0], ctypes.byref(o),
                                ctypes.byref(h)))
        else:
            _check(lib.eri_plan_mixed(sh, ns, ctypes.byref(b), q.ctypes.data, q.shape[0], qb.ctypes.data,
                                      float(fp32_below if fp32_below is not None else 0.0), ctypes.byref(o),
                                      ctypes.byref(h)))
        self._h = h
        self.nq = q.shape[0]
        self._keep = None

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            library().eri_plan_destroy(self._h)
            self._h = None

    @property
    def output_count(self) -> int:
        return int(library().eri_output_count(self._h))

    def offsets(self) -> np.ndarray:
        off = np.zeros(self.nq + 1, dtype=np.int64)
        _check(library().eri_output_offsets(self._h, off.ctypes.data))
        return off

    def stats(self) -> dict:
        s = np.zeros(8)
        _check(library().eri_plan_stats(self._h, s.ctypes.data, 8))
        return dict(launches=int(s[0]), flops=float(s[1]), scratch_bytes=float(s[2]), quartets=int(s[3]),
                    primitive_quartets=float(s[4]), h2d_bytes=float(s[5]), flops_fp32=float(s[6]),
                    fp32_parts=int(s[7]))

    def set_timing(self, enable=True):
        _check(library().eri_plan_set_timing(self._h, 1 if enable else 0))

    def launches(self):
        """Per-launch records of the last compute (call after the stream has
        completed): class, tier, grid, block, quartets, flops, ms, and for the
        cooperative tier the kind of contraction, the shape index (into
        class_shapes), the team size and the vote form."""
        lib = library()
        out = []
        for i in range(lib.eri_plan_launch_count(self._h)):
            info = np.zeros(8, dtype=np.int32)
            shp = np.zeros(4, dtype=np.int32)
            fl = ctypes.c_double()
            ms = ctypes.c_float()
            _check(lib.eri_plan_launch_info(self._h, i, info.ctypes.data, ctypes.byref(fl), ctypes.byref(ms)))
            _check(lib.eri_plan_launch_shape(self._h, i, shp.ctypes.data))
            out.append(dict(cls=tuple(int(x) for x in info[:4]), tier=int(info[4]), grid=int(info[5]),
                            block=int(info[6]), quartets=int(info[7]), flops=fl.value, ms=ms.value,
                            precision=int(lib.eri_plan_launch_precision(self._h, i)),
                            kind=KINDS_INV.get(int(shp[0])), shape=int(shp[1]), team=int(shp[2]),
                            votes={1: "off", 2: "on"}.get(int(shp[3]))))
        return out

    def compute(self, out, stream=None):
        """Write every block into ``out`` (a CUDA float64 tensor of at least
        output_count elements), asynchronously on ``stream``."""
        import torch
        if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64 and out.is_contiguous()):
            raise TypeError("out must be a contiguous CUDA float64 tensor")
        if out.numel() < self.output_count:
            raise ValueError("out is too small")
        _check(library().eri_compute(self._h, out.data_ptr(), _stream_handle(stream)))
        return out

    def compute_fixed_scratch(self, out, stream=None):
        """Like ``compute`` but without any device allocation: the kernels
        use the library's fixed 64 MiB scratch array (plans built with
        tier="global" only; see eri_compute_fixed_scratch)."""
        import torch
        if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64 and out.is_contiguous()):
            raise TypeError("out must be a contiguous CUDA float64 tensor")
        if out.numel() < self.output_count:
            raise ValueError("out is too small")
        _check(library().eri_compute_fixed_scratch(self._h, out.data_ptr(), _stream_handle(stream)))
        return out

    def schwarz(self, blocks, bounds, stream=None):
        """Schwarz factors Q_ab of an (ab|ab) plan from its computed blocks
        (both CUDA float64 tensors)."""
        _check(library().eri_schwarz(self._h, blocks.data_ptr(), bounds.data_ptr(), _stream_handle(stream)))
        return bounds

    def capture(self, out, stream):
        """Capture compute(out) on ``stream`` (not the default stream) into a
        CUDA graph; replay with ``replay``."""
        _check(library().eri_plan_graph_capture(self._h, out.data_ptr(), _stream_handle(stream)))

    def capture_jk(self, density, J, K, stream):
        """Capture compute_jk(density, J, K) on ``stream`` into a CUDA graph;
        each ``replay`` adds into J and K."""
        n = int(density.shape[0])
        _check(library().eri_plan_graph_capture_jk(self._h, self._square(density, n, "density"), n,
                                                   self._square(J, n, "J"), self._square(K, n, "K"),
                                                   _stream_handle(stream)))

    def replay(self, stream=None):
        _check(library().eri_plan_graph_launch(self._h, _stream_handle(stream)))

    @staticmethod
    def _square(t, n, name):
        import torch
        if t is None:
            return None
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and tuple(t.shape) == (n, n)):
            raise TypeError("{} must be a contiguous CUDA float64 tensor of shape ({n}, {n})".format(name, n=n))
        return t.data_ptr()

    def digest_jk(self, blocks, density, J=None, K=None, stream=None):
        """Add the Coulomb and exchange matrices of ``density`` from this
        plan's blocks into J and K (eri_digest_jk; plan built with
        digest=True)."""
        n = int(density.shape[0])
        _check(library().eri_digest_jk(self._h, blocks.data_ptr(), self._square(density, n, "density"), n,
                                       self._square(J, n, "J"), self._square(K, n, "K"), _stream_handle(stream)))

    def compute_jk(self, density, J=None, K=None, stream=None):
        """Evaluate and digest in one call (eri_compute_jk)."""
        n = int(density.shape[0])
        _check(library().eri_compute_jk(self._h, self._square(density, n, "density"), n, self._square(J, n, "J"),
                                        self._square(K, n, "K"), _stream_handle(stream)))

    def compute_host(self, out, stream=None):
        """Compute and copy every block into ``out`` (a contiguous CPU float64
        tensor, ideally pinned); asynchronous on ``stream``."""
        import torch
        if not (isinstance(out, torch.Tensor) and not out.is_cuda and out.dtype == torch.float64
                and out.is_contiguous()):
            raise TypeError("out must be a contiguous CPU float64 tensor")
        if out.numel() < self.output_count:
            raise ValueError("out is too small")
        _check(library().eri_compute_host(self._h, out.data_ptr(), _stream_handle(stream)))
        return out


def set_class_tier(ls, tier):
    """Process-wide preferred tier for class ls = (la, lb, lc, ld) (see the
    autotuner); tier name or 0 to clear."""
    t = TIERS[tier] if isinstance(tier, str) else int(tier)
    _check(library().eri_set_class_tier(*[int(x) for x in ls], t))


BOYS_FORMS = {"reg": 0, "coop": 1, "exec": 2}


def boys(T, L, form="coop", stream=None):
    """Device Boys values F_0..F_L at the arguments of the CUDA float64 tensor
    ``T`` (eri_boys_eval), as a tensor of shape (n, L + 1)."""
    import torch
    if not (isinstance(T, torch.Tensor) and T.is_cuda and T.dtype == torch.float64 and T.is_contiguous()):
        raise TypeError("T must be a contiguous CUDA float64 tensor")
    F = torch.empty((T.numel(), int(L) + 1), dtype=torch.float64, device=T.device)
    _check(library().eri_boys_eval(T.data_ptr(), T.numel(), int(L), BOYS_FORMS[form], F.data_ptr(),
                                   _stream_handle(stream)))
    return F


def screen_quartets(Q, pairs, threshold, stream=None):
    """Device Schwarz screening (eri_screen_quartets): Q a CUDA float64
    tensor [npair] of pair factors, pairs a CUDA int32 tensor [npair, 2];
    returns the surviving unique quartets as a CUDA int32 tensor [n, 4]."""
    import torch
    for t, dt in ((Q, torch.float64), (pairs, torch.int32)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError("Q must be a contiguous CUDA float64 tensor, pairs a contiguous CUDA int32 tensor")
    npair = Q.numel()
    if pairs.numel() != 2 * npair:
        raise ValueError("pairs must be [npair, 2]")
    lib = library()
    n = ctypes.c_int64()
    h = _stream_handle(stream)
    _check(lib.eri_screen_quartets(Q.data_ptr(), pairs.data_ptr(), npair, float(threshold), None, 0,
                                   ctypes.byref(n), h))
    out = torch.empty((max(1, n.value), 4), dtype=torch.int32, device=Q.device)
    _check(lib.eri_screen_quartets(Q.data_ptr(), pairs.data_ptr(), npair, float(threshold), out.data_ptr(),
                                   n.value, ctypes.byref(n), h))
    return out[: n.value]


KINDS = {"deep": 0, "shallow": 1, "single": 2}
KINDS_INV = {v: k for k, v in KINDS.items()}


def class_shapes(ls):
    """The cooperative shapes shipped for class ls (eri_class_shapes): a list
    of dicts (T, ilp, k1, k2, nslot); index 0 is the deep shape."""
    lib = library()
    n = lib.eri_class_shapes(*[int(x) for x in ls], None, 0)
    _check(min(n, 0))
    buf = (ctypes.c_int32 * max(1, 5 * n))()
    _check(min(lib.eri_class_shapes(*[int(x) for x in ls], buf, n), 0))
    return [dict(zip(("T", "ilp", "k1", "k2", "nslot"), buf[5 * i:5 * i + 5])) for i in range(n)]


def set_class_shape(ls, kind, shape, votes="auto"):
    """Process-wide preferred cooperative shape (an index into class_shapes,
    -1 clears) and vote form of class ls for one kind of contraction
    ("deep", "shallow", "single")."""
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    v = VOTES[votes] if isinstance(votes, str) else int(votes)
    _check(library().eri_set_class_shape(*[int(x) for x in ls], k, int(shape), v))


def set_class_votes(ls, votes):
    """Process-wide preferred cooperative form for class ls (autotuner):
    "off" (optional FP64 terms predicated per lane), "on" (skipped by warp
    vote), or "auto" / 0 to clear."""
    v = VOTES[votes] if isinstance(votes, str) else int(votes)
    _check(library().eri_set_class_votes(*[int(x) for x in ls], v))


def eri(basis, quartets, device="cuda", **opts):
    """Convenience: plan, compute on the current stream, return (values, offsets)."""
    import torch
    p = Plan(basis, quartets, **opts)
    out = torch.empty(max(1, p.output_count), dtype=torch.float64, device=device)
    p.compute(out)
    torch.cuda.current_stream().synchronize()
    off = p.offsets()
    p.close()
    return out[: off[-1]], off
