"""Differential walk on spheres for GB300 (sm_103a).

Importing the package loads nothing; ``paper_2405_12964_gb300.dwos`` loads the
CUDA library (``libdwos.so``, built in-tree) and raises if it is missing.
"""
__all__ = ["scenes", "dwos"]
