"""B300-native (sm_103a) FastVPINNs loss path: premultiplier tensors, tanh-MLP
forward with tangents, weak-residual contraction, variational + boundary +
sensor loss, and the adjoint back to the network weights and eps, behind the
C ABI of include/fastvpinn.h.

The CUDA library must be built (``python -m paper_2404_12063_b300.build``);
using the API without it raises.  There is no CPU fallback.
"""
import importlib

from ._native import FVError, LIB_PATH  # noqa: F401

_SUBMODULES = {"api", "build", "_native", "parallel"}


def __getattr__(name):
    if name in _SUBMODULES:
        return importlib.import_module("." + name, __name__)
    # the torch-based API is loaded lazily so that `build` works without torch/GPU
    api = importlib.import_module(".api", __name__)
    if hasattr(api, name):
        return getattr(api, name)
    raise AttributeError(name)
