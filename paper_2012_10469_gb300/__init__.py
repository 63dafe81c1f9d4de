"""GB300 (sm_103a) low-rank Matrix Exponentiated Gradient.

The method (Garber & Kaplan, Algorithm 2) runs in ``_lib/libmeg.so``,
built from ``csrc/`` by ``build.build()``; ``binding`` is its ctypes
front end.  Importing this package loads nothing.
"""
__all__ = ["binding", "build"]
