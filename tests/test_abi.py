"""Host-side checks of the C ABI: the library loads and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "helm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(helm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("helm_create", "helm_apply", "helm_vcycle", "helm_solve", "helm_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol():
    from paper_0912_0180_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_argument_errors_without_gpu():
    """Argument errors are detected on the host before any launch."""
    import paper_0912_0180_gb300 as P
    from paper_0912_0180_gb300 import _lib as L
    lib = P.load()
    assert lib.helm_status_str(0) == b"ok"
    out = ctypes.c_void_p()
    g = L.Grid()
    g.dim = 4  # invalid
    k = L.KSpec()
    pc = L.Precond()
    assert lib.helm_create(ctypes.byref(g), ctypes.byref(k), ctypes.byref(pc), None, ctypes.byref(out)) == L.HELM_ERR_ARG
    assert b"dim" in lib.helm_last_error()
    assert lib.helm_solve(None, None, None, None, None, None) == L.HELM_ERR_ARG
    assert lib.helm_apply(None, 1, None, None, None) == L.HELM_ERR_ARG
