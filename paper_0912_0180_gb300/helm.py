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
    vcycles: int = 0
    seconds: float = 0.0
    history_len: int = 0


def _info(ci, history=None) -> Info:
    return Info(ci.status, ci.iters, ci.matvecs, ci.restarts, ci.rel_res_recur, ci.rel_res_true, ci.kernels,
                history, ci.vcycles, ci.seconds, ci.history_len)


# ---- device memory: libhelm allocates through torch's caching allocator ---------------------
_keep = []        # every callback pair ever registered (blocks keep pointers to them)
_allocator = None  # None: nothing registered by this module yet; else "torch", "user" or "library"


def set_allocator(alloc=None, free=None):
    """helm_set_allocator with Python callables alloc(nbytes, stream) -> device pointer (int) or
    None, and free(ptr, stream); with no arguments, the library's own cudaMallocAsync.  The
    callbacks stay alive for the whole process: blocks allocated through them keep pointers to them
    and may be freed at any later time."""
    global _allocator
    lib = L.load()
    if alloc is None:
        lib.helm_set_allocator(L.ALLOC_FN(), L.FREE_FN(), None)
        _allocator = "library"
        return

    def _a(nbytes, stream, user):
        try:
            p = alloc(int(nbytes), int(stream or 0))
            return int(p) if p else None
        except Exception:  # any failure reads as out of memory: the library returns HELM_ERR_OOM
            return None

    def _f(ptr, stream, user):
        try:
            free(int(ptr), int(stream or 0))
        except Exception:
            pass

    cbs = (L.ALLOC_FN(_a), L.FREE_FN(_f))
    for cb in cbs:  # never collected, even at interpreter shutdown
        C.pythonapi.Py_IncRef(C.py_object(cb))
    _keep.append(cbs)
    lib.helm_set_allocator(cbs[0], cbs[1], None)
    _allocator = "user"


def use_torch_allocator(force: bool = False):
    """Route libhelm's device allocations through torch's caching allocator, on the stream the
    library allocates on.  The first context, server or parameter choice this module creates does
    this, unless set_allocator() chose another allocator before; force=True registers it anyway."""
    global _allocator
    if _allocator is not None and not force:
        return

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(max(nbytes, 1), torch.cuda.current_device(), stream)

    def free(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    set_allocator(alloc, free)
    _allocator = "torch"


def _grid(problem) -> "L.Grid":
    g = L.Grid()
    g.dim = problem.dim
    for a in range(3):
        g.n_int[a] = problem.n_int[a]
        g.n_layer[a][0], g.n_layer[a][1] = problem.n_layer[a]
        g.extent[a] = problem.extent[a]
    g.theta_gamma = problem.theta_gamma
    g.ecs_ramp = getattr(problem, "ecs_ramp", 0)
    return g


def _kspec(problem):
    """The k specification and the host arrays it points to (keep them alive while in use)."""
    k = L.KSpec()
    k.k0 = problem.k0
    keep = []
    if problem.phi is not None:
        phi = np.ascontiguousarray(problem.phi, dtype=np.float64)
        k.phi = phi.ctypes.data
        keep.append(phi)
    if getattr(problem, "phi_im", None) is not None:
        im = np.ascontiguousarray(problem.phi_im, dtype=np.float64)
        k.phi_im = im.ctypes.data
        keep.append(im)
    return k, keep


def _precond(precond, mg_dtype: str = "c64", flags: int = 0) -> "L.Precond":
    return L.Precond(precond.kind, precond.theta_beta, complex(precond.shift).real,
                     complex(precond.shift).imag, precond.nu1, precond.nu2, precond.smoother,
                     precond.omega, precond.max_levels, precond.coarse_max,
                     L.HELM_C64 if mg_dtype == "c64" else L.HELM_C128,
                     flags | (L.HELM_PF_GALERKIN if getattr(precond, "galerkin", False) else 0))


class Helm:
    """One instance: grid, ECS layers, k(x), the FP64 operator H and a preconditioner hierarchy.

    problem: helm_inputs.Problem; precond: helm_inputs.Precond; mg_dtype: "c64" (FP32 V-cycle)
    or "c128" (FP64 V-cycle).  Vectors are torch complex tensors on the current CUDA device.
    """

    def __init__(self, problem, precond, mg_dtype: str = "c64", stream=None, fused: bool = True,
                 pdl: bool = True, autotune: bool = True, k_field: Optional[torch.Tensor] = None,
                 k_bump: Optional[dict] = None):
        lib = L.load()
        self._lib = lib
        use_torch_allocator()
        g = _grid(problem)
        k, self._phi = _kspec(problem)
        if k_field is not None:  # k(x) as a device field (HELM_K_FIELD) instead of the problem's phi
            k.phi = k.phi_im = None
            k.kind = L.HELM_K_FIELD
            k.field = k_field.data_ptr()
            self._phi = [k_field]
        elif k_bump is not None:  # k0 (1 + amp exp(-|x - centre|^2 / width2)) formed on the device
            k.phi = k.phi_im = None
            k.kind = L.HELM_K_GAUSS_BUMP
            k.amp, k.width2 = k_bump["amp"], k_bump["width2"]
            for a, v in enumerate(k_bump["centre"]):
                k.centre[a] = v
        pc = _precond(precond, mg_dtype, (0 if fused else L.HELM_PF_UNFUSED) | (0 if pdl else L.HELM_PF_NO_PDL)
                      | (0 if autotune else L.HELM_PF_NO_AUTOTUNE))
        self._pc = pc
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

    def vcycle(self, r: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None, dtype=None,
               precond=None) -> torch.Tensor:
        """z = one V-cycle on M (helm_vcycle); dtype (torch.complex64 / complex128) is z's type,
        default the hierarchy's; complex128 from an FP32 hierarchy is its widened output.
        precond: None, or a helm_inputs.Precond that must be the context's own."""
        dt = dtype if dtype is not None else (out.dtype if out is not None else self.mg_dtype)
        if out is None:
            out = torch.empty(self.n, dtype=dt, device=r.device)
        pc = None if precond is None else C.byref(_precond(precond, "c64" if self.mg_dtype == torch.complex64 else "c128",
                                                           self._pc.flags))
        hd = L.HELM_C64 if dt == torch.complex64 else L.HELM_C128
        _check(self._lib.helm_vcycle(self._h, pc, hd, _ptr(r), _ptr(out), C.c_void_p(_stream(stream))), "helm_vcycle")
        return out

    def level_op(self, op: int, lvl: int, a: Optional[torch.Tensor], b: Optional[torch.Tensor] = None,
                 out: Optional[torch.Tensor] = None, count: int = 1, stream=None):
        _check(self._lib.helm_level_op(self._h, op, lvl, _ptr(a), _ptr(b), _ptr(out), count,
                                       C.c_void_p(_stream(stream))), "helm_level_op")
        return out

    def mg_iterate(self, f: torch.Tensor, max_cycles: int = 20, reduction: float = 1e-6, stream=None):
        """Multigrid as a stationary solver of M u = f (helm_mg_iterate; FP64 hierarchy): returns
        (cycles or -1, u, per-cycle residual ratios)."""
        u = torch.empty_like(f)
        k = C.c_int(-1)
        hist = np.zeros(max_cycles, np.float64)
        _check(self._lib.helm_mg_iterate(self._h, _ptr(f), _ptr(u), max_cycles, reduction, C.byref(k),
                                         hist.ctypes.data, C.c_void_p(_stream(stream))), "helm_mg_iterate")
        ran = k.value if k.value > 0 else int(np.count_nonzero(hist))
        return k.value, u, hist[:ran].copy()

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
        h = hist[: info.history_len].cpu().numpy() if hist is not None else None
        return x, _info(info, h)


def solve_batch(instances, bs, *, method=0, s=4, tol: float = 1e-6, maxmv: int = 2000,
                max_restarts: int = 3, shadows=None, stream=None, xs=None):
    """helm_solve_batch: solve every (Helm instance, rhs) pair at once; returns (xs, infos).
    `method` and `s` are one value for all instances or a sequence of one per instance; `xs`
    (optional) receives the solutions."""
    lib = L.load()
    n = len(instances)
    if xs is None:
        xs = [torch.empty(h.n, dtype=torch.complex128, device=b.device) for h, b in zip(instances, bs)]
    methods = list(method) if isinstance(method, (list, tuple)) else [method] * n
    ss = list(s) if isinstance(s, (list, tuple)) else [s] * n
    opts = (L.SolveOpts * max(n, 1))()
    keep = []
    for i in range(n):
        o = L.SolveOpts(methods[i], ss[i], tol, maxmv, max_restarts, None, None, 0)
        if shadows is not None and shadows[i] is not None:
            arr = np.ascontiguousarray(shadows[i], dtype=np.complex128)
            keep.append(arr)
            o.shadow = arr.ctypes.data
        opts[i] = o
    infos = (L.SolveInfo * max(n, 1))()
    cs = (C.c_void_p * max(n, 1))(*[h._h.value for h in instances])
    bp = (C.c_void_p * max(n, 1))(*[b.data_ptr() for b in bs])
    xp = (C.c_void_p * max(n, 1))(*[x.data_ptr() for x in xs])
    st = lib.helm_solve_batch(cs, bp, xp, n, opts, infos, C.c_void_p(_stream(stream)))
    _check(st, "helm_solve_batch", (L.HELM_OK, L.HELM_ERR_BREAKDOWN, L.HELM_ERR_MAXIT, L.HELM_ERR_NAN))
    out = [_info(infos[i]) for i in range(n)]
    return xs, out


def solve_group(instances, bs, *, tol: float = 1e-6, maxmv: int = 2000, max_restarts: int = 3, stream=None,
                xs=None):
    """helm_solve_group: Bi-CGSTAB on every (Helm instance, rhs) pair as one group, each kernel of an
    iteration one launch over all instances; returns (xs, infos)."""
    lib = L.load()
    n = len(instances)
    if xs is None:
        xs = [torch.empty(h.n, dtype=torch.complex128, device=b.device) for h, b in zip(instances, bs)]
    o = L.SolveOpts(0, 4, tol, maxmv, max_restarts, None, None, 0)
    infos = (L.SolveInfo * max(n, 1))()
    cs = (C.c_void_p * max(n, 1))(*[h._h.value for h in instances])
    bp = (C.c_void_p * max(n, 1))(*[b.data_ptr() for b in bs])
    xp = (C.c_void_p * max(n, 1))(*[x.data_ptr() for x in xs])
    st = lib.helm_solve_group(cs, bp, xp, n, C.byref(o), infos, C.c_void_p(_stream(stream)))
    _check(st, "helm_solve_group", (L.HELM_OK, L.HELM_ERR_BREAKDOWN, L.HELM_ERR_MAXIT, L.HELM_ERR_NAN))
    return xs, [_info(infos[i]) for i in range(n)]


class Server:
    """helm_server_*: continuous-batching solve server (requests from host memory)."""

    def __init__(self, budget_bytes: int, max_active: int = 4, smallest_first: bool = False):
        self._lib = L.load()
        use_torch_allocator()
        h = C.c_void_p()
        _check(self._lib.helm_server_create(int(budget_bytes), int(max_active), C.byref(h)), "helm_server_create")
        self._h = h
        self._keep = {}
        if smallest_first:
            _check(self._lib.helm_server_set_policy(h, L.HELM_SERVE_SMALLEST_FIRST), "helm_server_set_policy")

    def submit(self, problem, precond, *, mg_dtype: str = "c64", method: int = 0, s: int = 4,
               tol: float = 1e-6, maxmv: int = 2000, max_restarts: int = 3, shadow=None, rhs=None) -> int:
        """Queues one request; `rhs` (nrhs x N complex128) replaces problem.b when given, and
        wait() then returns x with the same shape."""
        rq = L.Request()
        rq.grid = _grid(problem)
        rq.k, phi = _kspec(problem)  # the server copies the arrays at submission
        rq.pc = _precond(precond, mg_dtype)
        rq.opts = L.SolveOpts(method, s, tol, maxmv, max_restarts, None, None, 0)
        sh = None
        if shadow is not None:
            sh = np.ascontiguousarray(shadow, dtype=np.complex128)
            rq.opts.shadow = sh.ctypes.data
        b = np.ascontiguousarray(problem.b if rhs is None else rhs, dtype=np.complex128)
        x = np.zeros_like(b)
        rq.b = b.ctypes.data
        rq.x = x.ctypes.data
        rq.nrhs = 1 if b.ndim == 1 else int(b.shape[0])
        t = C.c_uint64()
        _check(self._lib.helm_server_submit(self._h, C.byref(rq), C.byref(t)), "helm_server_submit")
        self._keep[t.value] = x
        return t.value

    def wait(self, ticket: int):
        """Blocks until the request is done; returns (x, Info, latency_s)."""
        info = L.SolveInfo()
        lat = C.c_double()
        st = self._lib.helm_server_wait(self._h, ticket, C.byref(info), C.byref(lat))
        _check(st, "helm_server_wait", (L.HELM_OK, L.HELM_ERR_BREAKDOWN, L.HELM_ERR_MAXIT, L.HELM_ERR_NAN))
        x = self._keep.pop(ticket)
        return x, _info(info), lat.value

    def stats(self):
        q, a, u = C.c_int(), C.c_int(), C.c_size_t()
        self._lib.helm_server_stats(self._h, C.byref(q), C.byref(a), C.byref(u))
        return q.value, a.value, u.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.helm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def select_precond(problem, start, f: torch.Tensor, max_cycles: int = 20, reduction: float = 1e-6,
                   factor: float = 0.8, max_trials: int = 16, stream=None):
    """Automatic CSL shift / CSG angle (helm_select_precond): returns (the chosen preconditioner
    as a helm_inputs.Precond, status, per-trial parameters, per-trial cycles)."""
    import dataclasses
    lib = L.load()
    use_torch_allocator()
    g = _grid(problem)
    k, phi = _kspec(problem)
    pc = _precond(start, "c128")
    out = L.Precond()
    params = np.zeros(max_trials, np.float64)
    cycles = np.zeros(max_trials, np.int32)
    trials = C.c_int(0)
    st = lib.helm_select_precond(C.byref(g), C.byref(k), C.byref(pc), _ptr(f), max_cycles, reduction, factor,
                                 max_trials, C.byref(out), params.ctypes.data, cycles.ctypes.data, C.byref(trials),
                                 C.c_void_p(_stream(stream)))
    _check(st, "helm_select_precond", ok=(L.HELM_OK, L.HELM_ERR_MAXIT))
    del phi
    if start.kind == 1:  # HELM_PC_CSL: the parameter is the imaginary shift
        chosen = dataclasses.replace(start, shift=complex(complex(start.shift).real, out.shift_im))
    else:
        chosen = dataclasses.replace(start, theta_beta=out.theta_beta)
    t = trials.value
    return chosen, st, params[:t].copy(), cycles[:t].copy()


def estimate_bytes(problem, precond, mg_dtype: str = "c64", method: int = 0, s: int = 4) -> int:
    lib = L.load()
    g = _grid(problem)
    pc = _precond(precond, mg_dtype)
    o = L.SolveOpts(method, s, 1e-6, 1000, 3, None, None, 0)
    return int(lib.helm_estimate_bytes(C.byref(g), C.byref(pc), C.byref(o)))
