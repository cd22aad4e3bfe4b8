"""GB300-native (sm_103a) mapping hot path of MonoGS++ (arXiv 2504.02437).

The differentiable 3D Gaussian splatting forward/backward, the L1 + planar loss,
Adam, dynamic insertion and densification, implemented as hand-written CUDA
behind the C ABI of ``include/gs.h``. Importing the package does not load the
library; ``GaussianMap`` does, and fails if the library is not built.
"""
from .build import build as build_library  # noqa: F401


def __getattr__(name):
    if name in ("GaussianMap", "MLP", "rasterize", "to_gs_camera", "default_config"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
