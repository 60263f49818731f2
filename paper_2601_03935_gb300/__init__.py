"""GB300 (sm_103a) library for the general synthetic iterative scheme (GSIS).

The compute lives in ``libgsis.so`` (CUDA, built in-tree by :mod:`.build`); the
``gsis`` module is a ctypes binding with the C entry points' names.
"""
from . import build  # noqa: F401
