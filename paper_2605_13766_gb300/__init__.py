"""GB300-native (sm_103a) FP64 Cosserat-rod step: CUDA library + thin Python binding.

``RodSystem`` wraps the C ABI of ``include/rod.h`` (librod.so).  The library is built
in-tree by ``paper_2605_13766_gb300.build.build()``; using the package without it raises.
"""
from .binding import LIBRARY_PATH, RodError, RodSystem, Surrogate, exported_symbols, load_library  # noqa: F401

__all__ = ["RodSystem", "Surrogate", "RodError", "load_library", "exported_symbols", "LIBRARY_PATH"]
