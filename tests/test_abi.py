"""The C-ABI library builds, loads and exports every entry point that
include/eri.h declares; error paths that need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eri.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eri_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_10312_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("eri_plan", "eri_compute", "eri_output_count", "eri_output_offsets", "eri_plan_destroy",
              "eri_last_error", "eri_compute_host", "eri_plan_stats"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_registry_and_blob_present(lib):
    from paper_2605_10312_gb300 import build
    assert os.path.exists(os.path.join(os.path.dirname(build.LIB), "eri_programs.bin"))
    n = ctypes.c_int.in_dll(lib, "eri_reg_count").value
    assert n > 0


def test_argument_errors_without_gpu():
    """Validation happens before any CUDA call, so these run on the CPU."""
    import numpy as np
    from paper_2605_10312_gb300 import eri, synth
    basis, q = synth.tiny_set()
    bad = synth.Basis(basis.centers, basis.shell_l.copy(), basis.shell_nprim, basis.shell_center,
                      basis.shell_prim, basis.exps, basis.coefs)
    bad.shell_l[0] = 5
    with pytest.raises(eri.EriError) as e:
        eri.Plan(bad, q[:4])
    assert e.value.code == -2
    with pytest.raises(eri.EriError) as e:
        eri.Plan(basis, np.array([[0, 1, 2, 99]]))
    assert e.value.code == -1
    neg = synth.Basis(basis.centers, basis.shell_l, basis.shell_nprim, basis.shell_center, basis.shell_prim,
                      -basis.exps, basis.coefs)
    with pytest.raises(eri.EriError) as e:
        eri.Plan(neg, q[:4])
    assert e.value.code == -1
    # launches take their quartet count as int32: 2^31 quartets are refused
    # before the quartet array is read
    lib = eri.library()
    sh, ns, b, keep = eri._marshal_basis(basis)
    qq = np.ascontiguousarray(q[:1])
    h = ctypes.c_void_p()
    assert lib.eri_plan(sh, ns, ctypes.byref(b), qq.ctypes.data, 1 << 31, None, ctypes.byref(h)) == -1
    assert b"too many quartets" in lib.eri_last_error()
    # an empty quartet list is a valid plan with no output
    p = eri.Plan(basis, np.zeros((0, 4), dtype=np.int32))
    assert p.output_count == 0
    p.close()


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """The binding has no CPU fallback: without the built library it raises."""
    import importlib
    from paper_2605_10312_gb300 import eri
    monkeypatch.setattr(eri, "_lib", None)
    with pytest.raises(RuntimeError):
        eri.library(str(tmp_path / "liberi.so"))
    importlib.reload(eri)
