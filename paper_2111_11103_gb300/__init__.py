"""GB300 (sm_103a) label fusion in semantically textured meshes (arXiv 2111.11103).

The compute path lives in ``liblabelfuse.so`` (hand-written CUDA kernels behind
the C ABI of ``include/labelfuse.h``); :mod:`.labelfuse` is its thin ctypes
binding.  Importing the package does not load the library; the first call
does, and fails loudly if it has not been built.
"""
from . import labelfuse  # noqa: F401
from .labelfuse import LabelFuseError, lib  # noqa: F401
