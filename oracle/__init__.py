"""CPU FP64 oracle for the DEC 0-form geometric-multigrid solver.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
CUDA library never links or calls it, and it shares no code with the CUDA
path: it is a plain, slow, readable restatement of what the paper defines,
in numpy/scipy, float64 throughout.

Modules
  mesh       embedded simplicial complex, signed incidence d0/d1, 1->4 subdivision
  dec        circumcentric Hodge stars and the 0-form Laplacian  L = *0^-1 d0^T *1 d0
  multigrid  interpolation M(f), restriction (row-normalized transpose), smoothers,
             V-cycle, coarse dense solve, standalone MG, flexible MG-PCG
  adjoint    adjoint solve and gradients with respect to b and *1
  porous     one explicit porous-convection step and its adjoint
  rk         adaptive Tsitouras 5(4) integration (the Tsit5 method of Sec. 3.2.2)

Parity pins live in tests/test_oracle_*.py.  Functions without an external
pin say "parity unpinned" in their docstring.
"""
