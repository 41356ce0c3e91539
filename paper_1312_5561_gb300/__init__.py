"""GB300-native solid Newton step of the partitioned FSI method of
Langer & Yang (arXiv:1312.5561): residual and consistent tangent of the
residual-stabilised P1/P1 u-p tetrahedral formulation (modified Mooney-Rivlin
and two-layer artery), 4x4 block-CSR assembly, and an AMG-preconditioned
Krylov solve, all in hand-written sm_103a CUDA behind the C ABI of
include/fsi_solid.h.

``from paper_1312_5561_gb300 import binding`` loads libfsi_solid.so (built
by ``paper_1312_5561_gb300.build``); there is no CPU fallback.
"""

__all__ = ["binding", "build"]


def __getattr__(name):
    if name in ("binding", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
