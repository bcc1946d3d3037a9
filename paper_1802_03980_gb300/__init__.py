"""GB300 camera tracking: IMU-seeded, median-filtered, orientation-regularised
coarse-to-fine point-to-plane ICP (arXiv 1802.03980) as CUDA kernels for sm_103a.

The C ABI is declared in include/kf_track.h and implemented by libkftrack.so
(built in-tree by ``build.build()``). Attribute access such as
``paper_1802_03980_gb300.kf_align`` loads the library and raises ImportError
when it has not been built: there is no other implementation to fall back to.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name.startswith("kf_") or name.startswith("KF_") or name in ("KFError", "load", "LIB_PATH"):
        from . import _lib
        return getattr(_lib, name)
    raise AttributeError(name)
