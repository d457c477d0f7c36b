"""ctypes declarations mirroring include/helm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhelm.so")

HELM_OK, HELM_ERR_ARG, HELM_ERR_OOM, HELM_ERR_CUDA = 0, 1, 2, 3
HELM_ERR_BREAKDOWN, HELM_ERR_MAXIT, HELM_ERR_NAN, HELM_ERR_TIMEOUT, HELM_ERR_BUSY = 4, 5, 6, 7, 8
HELM_C64, HELM_C128 = 0, 1
HELM_OP_APPLY, HELM_OP_RESIDUAL, HELM_OP_SMOOTH, HELM_OP_SMOOTH0 = 0, 1, 2, 3
HELM_OP_RESTRICT, HELM_OP_PROLONG, HELM_OP_COARSE, HELM_OP_DOWN = 4, 5, 6, 7
HELM_OP_TO_STORED, HELM_OP_FROM_STORED, HELM_OP_STORED = 8, 9, 0x100
HELM_PF_UNFUSED, HELM_PF_NO_PDL, HELM_PF_NO_AUTOTUNE, HELM_PF_GALERKIN = 1, 2, 4, 8
HELM_SERVE_FIFO, HELM_SERVE_SMALLEST_FIRST = 0, 1
HELM_K_CONST, HELM_K_GAUSS_BUMP, HELM_K_FIELD = 0, 1, 2

# helm_set_allocator callbacks: alloc(bytes, stream, user) -> device pointer or NULL;
# free(ptr, stream, user)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_int", C.c_int * 3), ("n_layer", (C.c_int * 2) * 3),
                ("extent", C.c_double * 3), ("theta_gamma", C.c_double),
                ("ecs_ramp", C.c_int)]


class KSpec(C.Structure):
    _fields_ = [("k0", C.c_double), ("phi", C.c_void_p), ("phi_im", C.c_void_p), ("kind", C.c_int),
                ("amp", C.c_double), ("width2", C.c_double), ("centre", C.c_double * 3),
                ("field", C.c_void_p)]


class Precond(C.Structure):
    _fields_ = [("kind", C.c_int), ("theta_beta", C.c_double), ("shift_re", C.c_double),
                ("shift_im", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int), ("smoother", C.c_int),
                ("omega", C.c_double), ("max_levels", C.c_int), ("coarse_max", C.c_int),
                ("mg_dtype", C.c_int), ("flags", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("method", C.c_int), ("s", C.c_int), ("tol", C.c_double), ("maxmv", C.c_int),
                ("max_restarts", C.c_int), ("shadow", C.c_void_p), ("history", C.c_void_p),
                ("host_loop", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("matvecs", C.c_int), ("restarts", C.c_int),
                ("rel_res_recur", C.c_double), ("rel_res_true", C.c_double), ("kernels", C.c_long),
                ("vcycles", C.c_int), ("seconds", C.c_double), ("history_len", C.c_int)]


class Request(C.Structure):
    _fields_ = [("grid", Grid), ("k", KSpec), ("pc", Precond), ("opts", SolveOpts), ("b", C.c_void_p),
                ("x", C.c_void_p), ("nrhs", C.c_int)]


_lib = None


def load() -> C.CDLL:
    """Load libhelm.so; raise if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhelm.so not built at {LIB_PATH}: run `python -m paper_0912_0180_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    vp, ip = C.c_void_p, C.c_int
    lib.helm_create.argtypes = [C.POINTER(Grid), C.POINTER(KSpec), C.POINTER(Precond), vp, C.POINTER(vp)]
    lib.helm_create.restype = ip
    lib.helm_size.argtypes = [vp]
    lib.helm_size.restype = C.c_long
    lib.helm_workspace_bytes.argtypes = [vp]
    lib.helm_workspace_bytes.restype = C.c_size_t
    lib.helm_num_levels.argtypes = [vp]
    lib.helm_num_levels.restype = ip
    lib.helm_level_shape.argtypes = [vp, ip, C.POINTER(C.c_int)]
    lib.helm_level_shape.restype = ip
    lib.helm_apply.argtypes = [vp, ip, vp, vp, vp]
    lib.helm_apply.restype = ip
    lib.helm_vcycle.argtypes = [vp, C.POINTER(Precond), ip, vp, vp, vp]
    lib.helm_vcycle.restype = ip
    lib.helm_level_op.argtypes = [vp, ip, ip, vp, vp, vp, ip, vp]
    lib.helm_level_op.restype = ip
    lib.helm_solve.argtypes = [vp, vp, vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo), vp]
    lib.helm_solve.restype = ip
    lib.helm_solve_batch.argtypes = [vp, vp, vp, ip, C.POINTER(SolveOpts), C.POINTER(SolveInfo), vp]
    lib.helm_solve_batch.restype = ip
    lib.helm_solve_group.argtypes = [vp, vp, vp, ip, C.POINTER(SolveOpts), C.POINTER(SolveInfo), vp]
    lib.helm_solve_group.restype = ip
    lib.helm_estimate_bytes.argtypes = [C.POINTER(Grid), C.POINTER(Precond), C.POINTER(SolveOpts)]
    lib.helm_estimate_bytes.restype = C.c_size_t
    lib.helm_server_create.argtypes = [C.c_size_t, ip, C.POINTER(vp)]
    lib.helm_server_create.restype = ip
    lib.helm_server_set_policy.argtypes = [vp, ip]
    lib.helm_server_set_policy.restype = ip
    lib.helm_server_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]
    lib.helm_server_submit.restype = ip
    lib.helm_server_poll.argtypes = [vp, C.c_uint64, C.POINTER(SolveInfo), C.POINTER(C.c_double)]
    lib.helm_server_poll.restype = ip
    lib.helm_server_wait.argtypes = [vp, C.c_uint64, C.POINTER(SolveInfo), C.POINTER(C.c_double)]
    lib.helm_server_wait.restype = ip
    lib.helm_server_stats.argtypes = [vp, C.POINTER(ip), C.POINTER(ip), C.POINTER(C.c_size_t)]
    lib.helm_server_stats.restype = ip
    lib.helm_server_destroy.argtypes = [vp]
    lib.helm_server_destroy.restype = None
    lib.helm_residual_noalloc.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.helm_residual_noalloc.restype = ip
    dp = C.c_double
    lib.helm_mg_iterate.argtypes = [vp, vp, vp, ip, dp, C.POINTER(ip), vp, vp]
    lib.helm_mg_iterate.restype = ip
    lib.helm_select_precond.argtypes = [C.POINTER(Grid), C.POINTER(KSpec), C.POINTER(Precond), vp, ip, dp, dp, ip,
                                        C.POINTER(Precond), vp, vp, C.POINTER(ip), vp]
    lib.helm_select_precond.restype = ip
    lib.helm_destroy.argtypes = [vp]
    lib.helm_destroy.restype = None
    lib.helm_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
    lib.helm_set_allocator.restype = None
    lib.helm_status_str.argtypes = [ip]
    lib.helm_status_str.restype = C.c_char_p
    lib.helm_last_error.argtypes = []
    lib.helm_last_error.restype = C.c_char_p
    _lib = lib
    return lib
