"""GB300-native RAS-PML solver for the 2D high-frequency Helmholtz equation.

The one-level restricted additive Schwarz preconditioner with PML
transmission conditions (RAS-PML) of Xie, Gong, Graham, Spence and Zhang,
inside a device-side flexible GMRES, for P1 finite elements. The compute path
is libraspml.so (hand-written CUDA for sm_103a, C ABI in include/raspml.h);
this package only marshals arguments to it.
"""
from ._lib import SYMBOLS, RasPmlError, load  # noqa: F401

__all__ = ["RasPml", "BatchRasPml", "load", "RasPmlError", "SYMBOLS", "build"]


def build(force: bool = False, verbose: bool = False) -> str:
    from .buildlib import build as _build
    return _build(force=force, verbose=verbose)


def __getattr__(name):
    if name == "RasPml":
        from .solver import RasPml
        return RasPml
    if name == "BatchRasPml":
        from .batch import BatchRasPml
        return BatchRasPml
    raise AttributeError(name)
