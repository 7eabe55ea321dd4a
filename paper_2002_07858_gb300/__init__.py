"""GB300-native Feldman-Cousins grid fit (arXiv 2002.07858): C-ABI CUDA library + thin binding.

The computation lives in ``csrc/`` (CUDA for sm_103a, exported through
``include/fc.h``); ``binding`` marshals arguments to it by ctypes.
"""
from .binding import *  # noqa: F401,F403
from .binding import FCError, load, lib_path  # noqa: F401

__all__ = [n for n in dir() if n.startswith(("fc_", "FC_"))] + ["FCError", "load", "lib_path"]
