"""GB300-native geometric multigrid for the DEC 0-form Laplacian (libdec).

The compute path is the CUDA library ``libdec.so`` built from ``csrc/`` for
sm_103a; this package only marshals arguments to its C ABI.  The public
names load the library on first use and raise ImportError if it has not been
built (``python -m paper_2508_12501_gb300.build``): there is no fallback.
"""

_EXPORTS = {"Hierarchy": "api", "Mesh": "api", "SolveStats": "api", "poisson_solve": "api", "Batch": "api",
            "BatchStats": "api", "tune_batch": "api",
            "DecError": "_lib"}

__all__ = sorted(_EXPORTS)


def __getattr__(name):
    mod = _EXPORTS.get(name)
    if mod is None:
        raise AttributeError(name)
    import importlib
    return getattr(importlib.import_module(f".{mod}", __name__), name)
