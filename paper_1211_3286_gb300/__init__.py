"""GB300 (sm_103a) relativistic lattice Boltzmann library for the scheme of
arXiv 1211.3286: a C-ABI CUDA library (librlb) and its thin Python binding.

Submodules: ``_lib`` (ctypes binding, same names as include/rlb.h), ``lattice``
(torch-facing handle wrapper), ``inputs`` (seeded synthetic fields), ``build``
(in-tree nvcc build)."""
from . import _lib  # noqa: F401
