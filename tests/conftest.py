import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    # build the in-tree library (git-ignored) and the oracle's C part
    import shutil
    from oracle.build import build as build_oracle
    build_oracle()
    if shutil.which("nvcc"):
        from paper_2512_04389_b300.build import build as build_lib
        build_lib()


def brute_fill(P):
    """Boolean Gaussian elimination without pivoting on a dense pattern:
    at step k every (i, j) with i, j > k, P[i, k] and P[k, j] becomes set."""
    import numpy as np
    P = P.copy().astype(bool)
    n = P.shape[0]
    for k in range(n):
        P[k + 1:, k + 1:] |= np.outer(P[k + 1:, k], P[k, k + 1:])
    return P


def random_sym_pattern(n, density, rng):
    import numpy as np
    M = rng.random((n, n)) < density
    M = M | M.T
    np.fill_diagonal(M, True)
    return M


def dense_to_csc(D, pattern=None):
    import numpy as np
    n = D.shape[0]
    if pattern is None:
        pattern = D != 0
    cols, rows = np.nonzero(pattern.T)
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(colptr, cols + 1, 1)
    colptr = np.cumsum(colptr)
    return colptr, rows.astype(np.int32), D[rows, cols].astype(np.float64)


@pytest.fixture(scope="session")
def rng():
    import numpy as np
    return np.random.Generator(np.random.PCG64(12345))
