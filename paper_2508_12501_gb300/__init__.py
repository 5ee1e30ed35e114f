"""GB300-native geometric multigrid for the DEC 0-form Laplacian (libdec).

The compute path is the CUDA library ``libdec.so`` built from ``csrc/`` for
sm_103a; this package only marshals arguments to its C ABI.  Importing it
fails if the library has not been built.
"""
from .api import Hierarchy, Mesh, SolveStats  # noqa: F401
from ._lib import DecError  # noqa: F401
