"""gbstencil: explicit finite-difference stencil sweeps (heat, acoustic wave) on GB300.

The computation lives in the CUDA library ``libgbstencil.so`` built from
``csrc/`` for sm_103a; :mod:`.native` binds its C ABI one-to-one and
:class:`.grid.Grid` wraps one handle with PyTorch supplying device memory and
streams.  Importing this package does not load CUDA; the first call does, and
fails loudly if the library cannot be built or loaded.
"""
from . import native  # noqa: F401
from .native import GbstError  # noqa: F401


def Grid(*args, **kwargs):  # noqa: N802 - factory keeps torch import lazy
    from .grid import Grid as _G
    return _G(*args, **kwargs)
