"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds input data only: base meshes (coordinates and triangle
lists) and seeded right-hand sides, fields and directions.  It contains none
of the method's arithmetic (no subdivision, Hodge stars, Laplacian, transfer
or solver step), so that the CUDA path and the CPU oracle can both consume
the same inputs while sharing no code.
"""
from .generators import *  # noqa: F401,F403
