"""FP64 CPU oracle for the spectral SOG quasi-2D Coulomb summation.

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py`` and by
nothing else; the CUDA library and its Python binding never load it, and it
never loads them.  Its results are the expected values of every parity test.

Modules:
  sog          the method step by step in numpy (Algorithms 1 and 2), the
               parameter selection of Sec. 4.3, and wrappers of the C sums.
  sog_oracle.c Ewald2D, brute-force image sums, the near-field direct sum and
               real-space Gaussian image sums, in plain C with OpenMP.

Every function is pinned by a ``-m "not gpu"`` test against something other
than itself (values printed in the paper, closed forms, limits, brute force);
see tests/test_oracle_*.py.
"""
from . import sog
from ._clib import build_oracle, num_threads

__all__ = ["sog", "build_oracle", "num_threads"]
