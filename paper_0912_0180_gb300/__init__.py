"""GB300-native ECS Helmholtz solver: CUDA kernels for sm_103a behind the C ABI in
include/helm.h (libhelm.so), with a thin torch/ctypes binding."""
from ._lib import LIB_PATH, load  # noqa: F401


def __getattr__(name):
    if name in ("Helm", "HelmError", "Info"):
        from . import helm as _h
        return getattr(_h, name)
    raise AttributeError(name)
