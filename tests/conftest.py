import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    import numpy as np
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#", ndmin=2)


_TB_EIG = {}


def tb_eig(n):
    """The tight-binding H of the bench sizes (seed 2000 + N) with its float64
    eigendecomposition (numpy/LAPACK), computed once per process and shared by the tests."""
    import numpy as np
    import synth
    if n not in _TB_EIG:
        h = synth.tight_binding(n, 2000 + n)
        w, u = np.linalg.eigh(h)
        _TB_EIG[n] = (h, w, u)
    return _TB_EIG[n]


def poly_columns(n, cols, c, ea, eb):
    """Columns `cols` of the oracle polynomial sum_j c_j T_j(X) of tb_eig(n)'s H on [ea, eb],
    from the eigendecomposition: U p(x(Lambda)) U^T e_j."""
    import numpy as np
    import oracle as O
    _, w, u = tb_eig(n)
    pw = np.polynomial.chebyshev.chebval(O.spectrum_scaled(w, ea, eb), c)
    return u @ (pw[:, None] * u[cols].T)


def header_symbols():
    """Function names declared in include/fermi.h."""
    import re
    path = os.path.join(ROOT, "include", "fermi.h")
    text = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fo_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="session")
def built_library():
    """Path of the shared library, building it in-tree if it is missing."""
    from paper_2306_12616_gb300 import build as B
    path = B.lib_path()
    if not os.path.exists(path):
        B.build()
    return path


@pytest.fixture(scope="session")
def solver(built_library):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_12616_gb300 import Solver
    s = Solver(0)
    yield s
    s.close()
