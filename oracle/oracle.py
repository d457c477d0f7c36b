"""ctypes marshalling for the C oracle (helm_oracle.c) -- test infrastructure only.

Every arithmetic step lives in helm_oracle.c; this file only builds it, loads it and moves
numpy arrays across.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "helm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB


def build_oracle(force: bool = False) -> str:
    """Compile helm_oracle.c into oracle/liboracle.so (portable flags, no FMA contraction), with
    OpenMP for its point-wise loops when the compiler has it (results are bitwise the same on
    any number of threads; without OpenMP the library is single-threaded)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-o", _LIB + ".tmp", _SRC, "-lm"]
            r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
            if r.returncode != 0:
                subprocess.run(base, check=True)
            os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def set_threads(n: int) -> int:
    """Threads for the oracle's point-wise loops (1 = serial); returns the previous count."""
    return int(_load().orc_set_threads(int(n)))


def get_threads() -> int:
    return int(_load().orc_get_threads())


class OracleError(RuntimeError):
    pass


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_int", C.c_int * 3), ("n_layer", (C.c_int * 2) * 3),
                ("extent", C.c_double * 3), ("theta_gamma", C.c_double),
                ("ecs_ramp", C.c_int)]


class _Precond(C.Structure):
    _fields_ = [("kind", C.c_int), ("theta_beta", C.c_double), ("shift_re", C.c_double),
                ("shift_im", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int),
                ("smoother", C.c_int), ("omega", C.c_double), ("max_levels", C.c_int),
                ("coarse_max", C.c_int), ("galerkin", C.c_int)]


class _Opts(C.Structure):
    _fields_ = [("method", C.c_int), ("s", C.c_int), ("tol", C.c_double), ("maxmv", C.c_int),
                ("max_restarts", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("matvecs", C.c_int),
                ("restarts", C.c_int), ("rel_res_recur", C.c_double), ("rel_res_true", C.c_double)]


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = C.CDLL(_LIB)
        vp, ip, dp = C.c_void_p, C.c_int, C.c_double
        lib.orc_create.restype = vp
        lib.orc_create.argtypes = [C.POINTER(_Grid), vp, vp, dp, C.POINTER(_Precond)]
        lib.orc_destroy.argtypes = [vp]
        lib.orc_num_levels.argtypes = [vp]
        lib.orc_level_shape.argtypes = [vp, ip, ip, vp]
        lib.orc_axis_tables.argtypes = [vp, ip, ip, ip, vp, vp, vp, vp, vp]
        lib.orc_level_phi.argtypes = [vp, ip, ip, vp, vp]
        lib.orc_level_st9.argtypes = [vp, ip, vp]
        lib.orc_level_st27.argtypes = [vp, ip, vp]
        lib.orc_apply.argtypes = [vp, ip, ip, vp, vp]
        lib.orc_dense.argtypes = [vp, ip, ip, vp]
        lib.orc_ilu_factors.argtypes = [vp, ip, vp]
        lib.orc_ilu_factors.restype = ip
        lib.orc_vcycle.argtypes = [vp, vp, vp]
        lib.orc_smooth.argtypes = [vp, ip, vp, vp, ip]
        lib.orc_restrict.argtypes = [vp, ip, vp, vp]
        lib.orc_prolong_add.argtypes = [vp, ip, vp, vp]
        lib.orc_coarse_solve.argtypes = [vp, vp, vp]
        lib.orc_dense_solve.argtypes = [vp, vp, vp]
        lib.orc_dense_solve.restype = ip
        lib.orc_solve.argtypes = [vp, vp, vp, C.POINTER(_Opts), vp, C.POINTER(_Info), vp, ip]
        lib.orc_solve.restype = ip
        lib.orc_mg_iterate.argtypes = [vp, vp, ip, dp, vp, vp]
        lib.orc_mg_iterate.restype = ip
        lib.orc_select_precond.argtypes = [C.POINTER(_Grid), vp, vp, dp, C.POINTER(_Precond), vp, ip, dp, dp, ip,
                                           C.POINTER(_Precond), vp, vp, C.POINTER(C.c_int)]
        lib.orc_select_precond.restype = ip
        lib.orc_set_threads.argtypes = [ip]
        lib.orc_set_threads.restype = ip
        lib.orc_get_threads.argtypes = []
        lib.orc_get_threads.restype = ip
        _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _grid(problem) -> "_Grid":
    g = _Grid()
    g.dim = problem.dim
    for a in range(3):
        g.n_int[a] = problem.n_int[a]
        g.n_layer[a][0] = problem.n_layer[a][0]
        g.n_layer[a][1] = problem.n_layer[a][1]
        g.extent[a] = problem.extent[a]
    g.theta_gamma = problem.theta_gamma
    g.ecs_ramp = getattr(problem, "ecs_ramp", 0)
    return g


def _phi_im(problem):
    """The imaginary part of phi (k at complex node positions), or None when phi is real."""
    v = getattr(problem, "phi_im", None)
    return None if v is None else np.ascontiguousarray(v, dtype=np.float64)


def _precond(pc) -> "_Precond":
    return _Precond(pc.kind, pc.theta_beta, complex(pc.shift).real, complex(pc.shift).imag,
                    pc.nu1, pc.nu2, pc.smoother, pc.omega, pc.max_levels, pc.coarse_max,
                    1 if getattr(pc, "galerkin", False) else 0)


def select_precond(problem, start, f, max_cycles=20, reduction=1e-6, factor=0.8, max_trials=16):
    """The parameter choice of Section 7's remark (orc_select_precond): returns the chosen
    parameter (CSL imaginary shift or CSG angle), the status (0 = the start converged) and, per
    trial, the parameter and the multigrid cycles it needed (-1 = did not converge)."""
    lib = _load()
    g = _grid(problem)
    p = _precond(start)
    phi = None if problem.phi is None else np.ascontiguousarray(problem.phi, dtype=np.float64)
    phi_im = _phi_im(problem)
    f = _c128(f)
    out = _Precond()
    params = np.zeros(max_trials, np.float64)
    cycles = np.zeros(max_trials, np.int32)
    status = C.c_int(0)
    t = lib.orc_select_precond(C.byref(g), _ptr(phi) if phi is not None else None,
                               _ptr(phi_im) if phi_im is not None else None, problem.k0, C.byref(p),
                               _ptr(f), max_cycles, reduction, factor, max_trials, C.byref(out),
                               _ptr(params), _ptr(cycles), C.byref(status))
    chosen = out.shift_im if start.kind == 1 else out.theta_beta
    return chosen, status.value, params[:t].copy(), cycles[:t].copy()


class Oracle:
    """One problem (grid + phi) with one preconditioner hierarchy."""

    H, M = 0, 1

    def __init__(self, problem, precond=None):
        from helm_inputs import Precond, PC_NONE
        lib = _load()
        self.problem = problem
        pc = precond if precond is not None else Precond(kind=PC_NONE)
        self.precond = pc
        g = _grid(problem)
        p = _precond(pc)
        self._phi = None
        if problem.phi is not None:
            self._phi = np.ascontiguousarray(problem.phi, dtype=np.float64)
        self._phi_im = _phi_im(problem)
        self._h = lib.orc_create(C.byref(g), _ptr(self._phi) if self._phi is not None else None,
                                 _ptr(self._phi_im) if self._phi_im is not None else None,
                                 problem.k0, C.byref(p))
        if not self._h:
            raise OracleError("singular coarsest preconditioner level (zero pivot in its dense LU)")
        self.n = problem.n
        self.nlev = lib.orc_num_levels(self._h)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_destroy(self._h)
            self._h = None

    def level_shape(self, which=1, lvl=0):
        out = np.zeros(3, np.int32)
        _lib.orc_level_shape(self._h, which, lvl, _ptr(out))
        return tuple(int(v) for v in out[: self.problem.dim])

    def level_size(self, which=1, lvl=0):
        return int(np.prod(self.level_shape(which, lvl)))

    def axis_tables(self, which, lvl, axis):
        n = self.level_shape(which, lvl)[axis]
        gap = np.zeros(n + 1, np.complex128)
        am, a0, ap = (np.zeros(n, np.complex128) for _ in range(3))
        pos = np.zeros(n, np.float64)
        _lib.orc_axis_tables(self._h, which, lvl, axis, _ptr(gap), _ptr(am), _ptr(a0), _ptr(ap), _ptr(pos))
        return dict(gap=gap, am=am, a0=a0, ap=ap, pos=pos)

    def level_phi(self, which, lvl):
        phi = np.zeros(self.level_size(which, lvl), np.float64)
        s = np.zeros(1, np.complex128)
        _lib.orc_level_phi(self._h, which, lvl, _ptr(phi), _ptr(s))
        return phi, complex(s[0])

    def level_stencil9(self, lvl):
        """Galerkin 9-point stencil of preconditioner level lvl, shape (ntot, 3, 3) indexed
        [p, dj+1, di+1]; zeros for a Shortley-Weller level."""
        m = self.level_size(1, lvl)
        out = np.zeros(9 * m, np.complex128)
        _lib.orc_level_st9(self._h, lvl, _ptr(out))
        return out.reshape(m, 3, 3)

    def level_stencil27(self, lvl):
        """Galerkin 27-point stencil of preconditioner level lvl (3D), shape (ntot, 3, 3, 3)
        indexed [p, dl+1, dj+1, di+1]; zeros for a Shortley-Weller level."""
        m = self.level_size(1, lvl)
        out = np.zeros(27 * m, np.complex128)
        _lib.orc_level_st27(self._h, lvl, _ptr(out))
        return out.reshape(m, 3, 3, 3)

    def apply(self, x, which=0, lvl=0):
        x = _c128(x)
        y = np.empty(self.level_size(which, lvl), np.complex128)
        _lib.orc_apply(self._h, which, lvl, _ptr(x), _ptr(y))
        return y

    def ilu_factors(self, lvl):
        """ILU(0) factors of preconditioner level lvl, shape (ntot, 3, 3) indexed [p, dj+1, di+1]
        like a Galerkin stencil: L at the lower neighbours (unit diagonal implied), U at p and its
        upper neighbours; None when the level has none (another smoother or the coarsest)."""
        m = self.level_size(1, lvl)
        out = np.zeros(9 * m, np.complex128)
        if not _lib.orc_ilu_factors(self._h, lvl, _ptr(out)):
            return None
        return out.reshape(m, 3, 3)

    def dense(self, which=0, lvl=0):
        m = self.level_size(which, lvl)
        A = np.zeros((m, m), np.complex128)
        _lib.orc_dense(self._h, which, lvl, _ptr(A))
        return A

    def vcycle(self, r):
        r = _c128(r)
        z = np.empty(self.n, np.complex128)
        _lib.orc_vcycle(self._h, _ptr(r), _ptr(z))
        return z

    def smooth(self, lvl, u, f, sweeps=1):
        u = _c128(u).copy()
        f = _c128(f)
        _lib.orc_smooth(self._h, lvl, _ptr(u), _ptr(f), sweeps)
        return u

    def restrict(self, lvl, r):
        r = _c128(r)
        fc = np.empty(self.level_size(1, lvl + 1), np.complex128)
        _lib.orc_restrict(self._h, lvl, _ptr(r), _ptr(fc))
        return fc

    def prolong_add(self, lvl, ec, u):
        ec = _c128(ec)
        u = _c128(u).copy()
        _lib.orc_prolong_add(self._h, lvl, _ptr(ec), _ptr(u))
        return u

    def coarse_solve(self, f):
        f = _c128(f)
        z = np.empty_like(f)
        _lib.orc_coarse_solve(self._h, _ptr(f), _ptr(z))
        return z

    def mg_iterate(self, f, max_cycles, reduction):
        """Multigrid as a stationary solver of M u = f from u = 0 (orc_mg_iterate): returns
        (cycles or -1, u, residual history)."""
        f = _c128(f)
        u = np.empty(self.n, np.complex128)
        hist = np.zeros(max_cycles, np.float64)
        k = _lib.orc_mg_iterate(self._h, _ptr(f), max_cycles, reduction, _ptr(u), _ptr(hist))
        ran = k if k > 0 else int(np.count_nonzero(hist))
        return k, u, hist[:ran].copy()

    def dense_solve(self, b):
        b = _c128(b)
        x = np.empty_like(b)
        rc = _lib.orc_dense_solve(self._h, _ptr(b), _ptr(x))
        if rc != 0:
            raise RuntimeError("singular operator")
        return x

    def solve(self, b, opts, shadow=None, history=False):
        b = _c128(b)
        x = np.zeros(self.n, np.complex128)
        o = _Opts(opts.method, opts.s, opts.tol, opts.maxmv, opts.max_restarts)
        info = _Info()
        sh = None
        if shadow is not None:
            sh = _c128(shadow)
            assert sh.shape == (opts.s, self.n)
        hist = np.zeros(opts.maxmv + 8, np.float64) if history else None
        _lib.orc_solve(self._h, _ptr(b), _ptr(x), C.byref(o), _ptr(sh) if sh is not None else None,
                       C.byref(info), _ptr(hist) if hist is not None else None,
                       len(hist) if hist is not None else 0)
        out = dict(status=info.status, iters=info.iters, matvecs=info.matvecs,
                   restarts=info.restarts, rel_res_recur=info.rel_res_recur,
                   rel_res_true=info.rel_res_true)
        if history:
            out["history"] = hist[: info.matvecs].copy()
        return x, out
