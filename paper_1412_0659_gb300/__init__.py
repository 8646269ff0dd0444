"""GB300-native (sm_103a) gravitational tree force after Bonsai (SC14).

The compute path is a C-ABI shared library of hand-written CUDA kernels
(``csrc/``, declared in ``include/bonsai_gb.h``); :mod:`.capi` is a thin
ctypes binding with the same names.  PyTorch supplies device memory and
streams only.  There is no CPU fallback: calls fail loudly when the CUDA
library is missing.
"""
from .flops import FLOPS_PC, FLOPS_PP, fp32_peak_tflops, tree_force_flops  # noqa: F401


def __getattr__(name):
    # the CUDA binding and the object wrapper load torch; import them on demand
    if name in ("capi", "gravity", "galaxy", "domains", "autograd"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    if name == "TreeGravity":
        from .gravity import TreeGravity
        return TreeGravity
    raise AttributeError(name)
