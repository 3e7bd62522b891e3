"""CPU FP64 oracle for the Chebyshev Fermi-operator expansion.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct restatement of
the method in numpy/LAPACK float64. Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library path never does, and the
library fails loudly when its CUDA extension is missing instead of falling back here.
It shares no code with the CUDA path: no kernels, headers, helpers, tables or constants.

Parity status of each function is listed in the module docstring of ``oracle.fermi``.
"""
from .fermi import *  # noqa: F401,F403
