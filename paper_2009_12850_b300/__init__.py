"""B300-native Piacsek-Williams advection source terms (su, sv, sw of u, v, w).

Modules (imported on first use so that importing the package needs neither a
GPU nor the built library):
  _lib       ctypes binding of the C-ABI library libpwadv.so (include/pwadv.h)
  api        Mesh and Batch: torch-facing wrappers (device memory, streams)
  autograd   PWAdvect / PWEulerSegment autograd functions and the checkpointed loop
  synthetic  seeded synthetic inputs shaped like the paper's runs
  build      nvcc build of libpwadv.so for sm_103a
"""
import importlib

__all__ = ["api", "autograd", "synthetic", "build"]


def __getattr__(name):
    if name in ("_lib", "api", "autograd", "synthetic", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
