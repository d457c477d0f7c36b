"""Python binding of the C ABI in include/helm.h: same entry points, torch tensors for device
memory and the current CUDA stream.  Every step of the solver runs in libhelm's kernels; this
module only marshals arguments."""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional

import numpy as np
import torch

from . import _lib as L


class HelmError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = L.load()
        msg = lib.helm_status_str(status).decode()
        detail = lib.helm_last_error().decode()
        super().__init__(f"{where}: {msg}" + (f" ({detail})" if detail else ""))
        self.status = status


def _check(status: int, where: str, ok=(L.HELM_OK,)):
    if status not in ok:
        raise HelmError(status, where)
    return status


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


@dataclasses.dataclass
class Info:
    status: int
    iters: int
    matvecs: int
    restarts: int
    rel_res_recur: float
    rel_res_true: float
    kernels: int = 0
    history: Optional[np.ndarray] = None


class Helm:
    """One instance: grid, ECS layers, k(x), the FP64 operator H and a preconditioner hierarchy.

    problem: helm_inputs.Problem; precond: helm_inputs.Precond; mg_dtype: "c64" (FP32 V-cycle)
    or "c128" (FP64 V-cycle).  Vectors are torch complex tensors on the current CUDA device.
    """

    def __init__(self, problem, precond, mg_dtype: str = "c64", stream=None, fused: bool = True,
                 pdl: bool = True):
        lib = L.load()
        self._lib = lib
        g = L.Grid()
        g.dim = problem.dim
        for a in range(3):
            g.n_int[a] = problem.n_int[a]
            g.n_layer[a][0], g.n_layer[a][1] = problem.n_layer[a]
            g.extent[a] = problem.extent[a]
        g.theta_gamma = problem.theta_gamma
        k = L.KSpec()
        k.k0 = problem.k0
        self._phi = None
        if problem.phi is not None:
            self._phi = np.ascontiguousarray(problem.phi, dtype=np.float64)
            k.phi = self._phi.ctypes.data
        pc = L.Precond(precond.kind, precond.theta_beta, complex(precond.shift).real,
                       complex(precond.shift).imag, precond.nu1, precond.nu2, precond.smoother,
                       precond.omega, precond.max_levels, precond.coarse_max,
                       L.HELM_C64 if mg_dtype == "c64" else L.HELM_C128,
                       (0 if fused else L.HELM_PF_UNFUSED) | (0 if pdl else L.HELM_PF_NO_PDL))
        h = C.c_void_p()
        _check(lib.helm_create(C.byref(g), C.byref(k), C.byref(pc), C.c_void_p(_stream(stream)), C.byref(h)),
               "helm_create")
        self._h = h
        self.problem = problem
        self.n = int(lib.helm_size(h))
        self.mg_dtype = torch.complex64 if mg_dtype == "c64" else torch.complex128
        self.nlev = int(lib.helm_num_levels(h))

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None):
            self._lib.helm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def workspace_bytes(self) -> int:
        return int(self._lib.helm_workspace_bytes(self._h))

    def level_shape(self, lvl: int):
        n = (C.c_int * 3)()
        _check(self._lib.helm_level_shape(self._h, lvl, n), "helm_level_shape")
        return tuple(int(v) for v in n[: self.problem.dim])

    # -- entry points --
    def apply(self, x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.n, dtype=torch.complex128, device=x.device)
        dt = L.HELM_C64 if x.dtype == torch.complex64 else L.HELM_C128
        _check(self._lib.helm_apply(self._h, dt, _ptr(x), _ptr(out), C.c_void_p(_stream(stream))), "helm_apply")
        return out

    def vcycle(self, r: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.n, dtype=self.mg_dtype, device=r.device)
        _check(self._lib.helm_vcycle(self._h, _ptr(r), _ptr(out), C.c_void_p(_stream(stream))), "helm_vcycle")
        return out

    def level_op(self, op: int, lvl: int, a: Optional[torch.Tensor], b: Optional[torch.Tensor] = None,
                 out: Optional[torch.Tensor] = None, count: int = 1, stream=None):
        _check(self._lib.helm_level_op(self._h, op, lvl, _ptr(a), _ptr(b), _ptr(out), count,
                                       C.c_void_p(_stream(stream))), "helm_level_op")
        return out

    def solve(self, b: torch.Tensor, x: Optional[torch.Tensor] = None, *, method: int = 0, s: int = 4,
              tol: float = 1e-6, maxmv: int = 2000, max_restarts: int = 3,
              shadow: Optional[np.ndarray] = None, stream=None, raise_on_error: bool = False,
              history: bool = False, host_loop: bool = False):
        """Solve H x = b from x = 0; returns (x, Info).  Krylov statuses (breakdown, cap, NaN) are
        reported in Info; CUDA and argument errors raise."""
        if x is None:
            x = torch.empty(self.n, dtype=torch.complex128, device=b.device)
        o = L.SolveOpts(method, s, tol, maxmv, max_restarts, None, None, 1 if host_loop else 0)
        hist = None
        if history:
            hist = torch.full((maxmv,), float("nan"), dtype=torch.float64, device=b.device)
            o.history = hist.data_ptr()
        if shadow is not None:
            self._shadow = np.ascontiguousarray(shadow, dtype=np.complex128)
            o.shadow = self._shadow.ctypes.data
        info = L.SolveInfo()
        st = self._lib.helm_solve(self._h, _ptr(b), _ptr(x), C.byref(o), C.byref(info),
                                  C.c_void_p(_stream(stream)))
        ok = (L.HELM_OK,) if raise_on_error else (L.HELM_OK, L.HELM_ERR_BREAKDOWN, L.HELM_ERR_MAXIT, L.HELM_ERR_NAN)
        _check(st, "helm_solve", ok)
        h = hist[: info.matvecs].cpu().numpy() if hist is not None else None
        return x, Info(info.status, info.iters, info.matvecs, info.restarts, info.rel_res_recur,
                       info.rel_res_true, info.kernels, h)
