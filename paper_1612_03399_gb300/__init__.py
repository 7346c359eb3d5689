"""GB300-native Lagrangian hot path of the interaction-potential + MLS
immersed-boundary method (Spandan et al., J. Comp. Phys.): internal forces,
MLS interpolation and probe traction, node update and spreading for many
triangulated bodies, as hand-written CUDA for sm_103a behind a C ABI
(include/ibm.h).  This package holds the in-tree build, the ctypes binding and
the seeded workload generators."""

__all__ = ["Context", "IBMError", "library", "build"]


def __getattr__(name):
    if name in ("Context", "IBMError", "library"):
        from . import _lib
        return getattr(_lib, name)
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
