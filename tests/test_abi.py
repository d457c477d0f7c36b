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


def test_argument_errors_of_the_newer_entry_points_without_gpu():
    """A side below -1, a bad ramp, ILU(0) on a 3D grid, an unknown smoother, GMRES restart lengths
    and the parameter choice's arguments are refused on the host (no device is touched)."""
    import helm_inputs as hi
    import paper_0912_0180_gb300 as P
    from paper_0912_0180_gb300 import _lib as L
    from paper_0912_0180_gb300.helm import _grid, _kspec, _precond
    lib = P.load()
    out = ctypes.c_void_p()
    p = hi.make_problem(2, 17, ((-2, 0), (0, 0)), k0=3.0, rhs="zero")  # a side below -1
    k, keep = _kspec(p)
    pc = _precond(hi.Precond(kind=hi.PC_NONE), "c128")
    assert lib.helm_create(ctypes.byref(_grid(p)), ctypes.byref(k), ctypes.byref(pc), None, ctypes.byref(out)) \
        == L.HELM_ERR_ARG
    q = hi.make_problem(2, 17, 4, k0=3.0, rhs="zero")
    g = _grid(q)
    g.ecs_ramp = -2
    k, keep = _kspec(q)
    assert lib.helm_create(ctypes.byref(g), ctypes.byref(k), ctypes.byref(pc), None, ctypes.byref(out)) \
        == L.HELM_ERR_ARG
    # phi_im without phi
    k = L.KSpec()
    k.k0 = 3.0
    im = (ctypes.c_double * q.n)()
    k.phi_im = ctypes.cast(im, ctypes.c_void_p)
    assert lib.helm_create(ctypes.byref(_grid(q)), ctypes.byref(k), ctypes.byref(pc), None, ctypes.byref(out)) \
        == L.HELM_ERR_ARG
    # ILU(0) smoothing on a 3D grid, and an unknown smoother kind
    c = hi.make_problem(3, 9, 2, k0=3.0, rhs="zero")
    k3, keep3 = _kspec(c)
    pi = _precond(hi.Precond(kind=hi.PC_CSG_UNIFORM, smoother=hi.SM_ILU), "c128")
    assert lib.helm_create(ctypes.byref(_grid(c)), ctypes.byref(k3), ctypes.byref(pi), None, ctypes.byref(out)) \
        == L.HELM_ERR_ARG
    assert b"ILU" in lib.helm_last_error()
    pu = _precond(hi.Precond(kind=hi.PC_CSG_UNIFORM, smoother=7), "c128")
    k, keep = _kspec(q)
    assert lib.helm_create(ctypes.byref(_grid(q)), ctypes.byref(k), ctypes.byref(pu), None, ctypes.byref(out)) \
        == L.HELM_ERR_ARG
    # the parameter choice: factor outside (0, 1), identity preconditioner
    k, keep = _kspec(q)
    sel_out = L.Precond()
    trials = ctypes.c_int(0)
    start = _precond(hi.Precond(kind=hi.PC_CSL), "c128")
    dummy = ctypes.c_void_p(16)  # never dereferenced: arguments are checked first
    assert lib.helm_select_precond(ctypes.byref(_grid(q)), ctypes.byref(k), ctypes.byref(start), dummy, 20, 1e-6,
                                   1.5, 8, ctypes.byref(sel_out), None, None, ctypes.byref(trials), None) \
        == L.HELM_ERR_ARG
    assert lib.helm_select_precond(ctypes.byref(_grid(q)), ctypes.byref(k), ctypes.byref(pc), dummy, 20, 1e-6,
                                   0.8, 8, ctypes.byref(sel_out), None, None, ctypes.byref(trials), None) \
        == L.HELM_ERR_ARG
    assert trials.value == 0


def test_memory_estimate_counts_galerkin_stencils_and_gmres_basis():
    """helm_estimate_bytes (host only) grows by the stored Galerkin stencils (27 weights per coarse
    unknown in 3D), by the GMRES(m) basis of m + 1 vectors and by the ILU(0) factors."""
    import helm_inputs as hi
    from paper_0912_0180_gb300.helm import estimate_bytes
    p = hi.make_problem(3, 66, 16, k0=10.0, rhs="zero")  # 80^3 unknowns
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, smoother=hi.SM_JACOBI)
    pg = hi.Precond(kind=hi.PC_CSG_UNIFORM, smoother=hi.SM_JACOBI, galerkin=True)
    base, gal = estimate_bytes(p, pc, "c128"), estimate_bytes(p, pg, "c128")
    n1 = 40 ** 3  # the first coarse level
    assert gal - base >= 27 * 16 * n1
    g30, g60 = estimate_bytes(p, pc, "c128", method=2, s=30), estimate_bytes(p, pc, "c128", method=2, s=60)
    assert g60 - g30 >= 30 * 16 * p.n
    # ILU(0) factors: 9 entries per unknown on every level above the coarsest (2D grid)
    p2 = hi.make_problem(2, 300, 20, k0=10.0, rhs="zero")
    pi = hi.Precond(kind=hi.PC_CSG_UNIFORM, smoother=hi.SM_ILU)
    pj = hi.Precond(kind=hi.PC_CSG_UNIFORM, smoother=hi.SM_JACOBI)
    assert estimate_bytes(p2, pi, "c64") - estimate_bytes(p2, pj, "c64") >= 9 * 24 * p2.n
