"""ctypes front of the C oracle: plain FP64 Gilbert-Peierls LU and solves.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .build import build

_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        lib.orc_lu_factor.argtypes = [C.c_int64, P, P, P, C.c_double,
                                      C.POINTER(P)]
        lib.orc_lu_factor.restype = C.c_int
        for f in ("orc_lu_n", "orc_lu_lnnz", "orc_lu_unnz", "orc_lu_nperturb"):
            getattr(lib, f).argtypes = [P]
            getattr(lib, f).restype = C.c_int64
        lib.orc_lu_copy.argtypes = [P] * 7
        lib.orc_lu_free.argtypes = [P]
        for f in ("orc_lsolve", "orc_usolve", "orc_ltsolve", "orc_utsolve"):
            getattr(lib, f).argtypes = [C.c_int64, P, P, P, P, C.c_int64,
                                        C.c_int32]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class SingularError(RuntimeError):
    pass


def symmetrize(n, colptr, rowidx, values):
    """Pattern of A + A^T plus the full diagonal, as CSC with sorted rows.

    Positions of A keep A's values; positions added by the symmetrization or
    the diagonal hold explicit zeros.  This is the structurally symmetric
    input that the paper's diagonal-block pointer assumes (Section 4.2).
    """
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    rows = rowidx.astype(np.int64)
    r = np.concatenate([rows, cols, np.arange(n)])
    c = np.concatenate([cols, rows, np.arange(n)])
    key = np.unique(c * n + r)
    sc = key // n
    sr = key % n
    sp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(sp, sc + 1, 1)
    sp = np.cumsum(sp)
    sv = np.zeros(key.size)
    pos = np.searchsorted(key, cols * n + rows)
    sv[pos] = values
    return sp, sr.astype(np.int32), sv


def lu(n, colptr, rowidx, values, tau=0.0, symmetric_pattern=True):
    """A = L U without row exchanges.  Returns a dict with CSC arrays
    Lp, Li, Lx (strictly lower; unit diagonal implied) and Up, Ui, Ux (upper
    incl. diagonal, last in each column), plus ``nperturb``.

    With ``symmetric_pattern`` the pattern of A + A^T (plus diagonal) is
    factored, so L's and U's patterns are transposes of each other.
    """
    if symmetric_pattern:
        colptr, rowidx, values = symmetrize(n, colptr, rowidx, values)
    ap = np.ascontiguousarray(colptr, dtype=np.int64)
    ai = np.ascontiguousarray(rowidx, dtype=np.int32)
    ax = np.ascontiguousarray(values, dtype=np.float64)
    lib = _L()
    h = C.c_void_p()
    rc = lib.orc_lu_factor(n, _p(ap), _p(ai), _p(ax), float(tau), C.byref(h))
    if rc == 2:
        raise SingularError("zero pivot with perturbation disabled")
    if rc != 0:
        raise RuntimeError(f"oracle LU failed: {rc}")
    try:
        ln = lib.orc_lu_lnnz(h)
        un = lib.orc_lu_unnz(h)
        F = dict(Lp=np.empty(n + 1, np.int64), Li=np.empty(ln, np.int32),
                 Lx=np.empty(ln), Up=np.empty(n + 1, np.int64),
                 Ui=np.empty(un, np.int32), Ux=np.empty(un))
        lib.orc_lu_copy(h, *(_p(F[k]) for k in
                             ("Lp", "Li", "Lx", "Up", "Ui", "Ux")))
        F["nperturb"] = int(lib.orc_lu_nperturb(h))
        F["n"] = n
    finally:
        lib.orc_lu_free(h)
    return F


def _solve(fn, n, p, i, x, B):
    X = np.array(B, dtype=np.float64, order="F", copy=True)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    getattr(_L(), fn)(n, _p(p), _p(i), _p(x), _p(X), X.shape[0],
                      X.shape[1])
    return X


def lsolve(F, B):
    """Solve L X = B (L unit lower)."""
    return _solve("orc_lsolve", F["n"], F["Lp"], F["Li"], F["Lx"], B)


def usolve(F, B):
    """Solve U X = B."""
    return _solve("orc_usolve", F["n"], F["Up"], F["Ui"], F["Ux"], B)


def ltsolve(F, B):
    """Solve L^T X = B."""
    return _solve("orc_ltsolve", F["n"], F["Lp"], F["Li"], F["Lx"], B)


def utsolve(F, B):
    """Solve U^T X = B."""
    return _solve("orc_utsolve", F["n"], F["Up"], F["Ui"], F["Ux"], B)


def solve(F, B):
    """x = A^{-1} b = U^{-1} L^{-1} b."""
    return usolve(F, lsolve(F, B))


def solve_transpose(F, G):
    """lambda = A^{-T} g = L^{-T} U^{-T} g."""
    return ltsolve(F, utsolve(F, G))


def lu_pattern(F):
    """Filled pattern of L + U (strict L, U incl. diagonal) as CSC with
    sorted rows, plus the values in that order."""
    n = F["n"]
    lc = np.repeat(np.arange(n, dtype=np.int64), np.diff(F["Lp"]))
    uc = np.repeat(np.arange(n, dtype=np.int64), np.diff(F["Up"]))
    r = np.concatenate([F["Ui"].astype(np.int64), F["Li"].astype(np.int64)])
    c = np.concatenate([uc, lc])
    v = np.concatenate([F["Ux"], F["Lx"]])
    o = np.lexsort((r, c))
    p = np.zeros(n + 1, dtype=np.int64)
    np.add.at(p, c + 1, 1)
    return np.cumsum(p), r[o].astype(np.int32), v[o]


def flops(F):
    """Algorithmic flop count of the factorization:
    sum_k (l_k + 2 l_k u_k), with l_k the stored strictly-lower entries of
    L(:,k) and u_k the strictly-upper entries of U(k,:) (Table 3 counts
    floating-point operations of the numerical factorization)."""
    n = F["n"]
    l = np.diff(F["Lp"]).astype(np.int64)
    ur = np.zeros(n, dtype=np.int64)
    uc = np.repeat(np.arange(n), np.diff(F["Up"]))
    strict = F["Ui"] != uc
    np.add.at(ur, F["Ui"][strict], 1)
    return int(np.sum(l + 2 * l * ur))


def matvec(n, colptr, rowidx, values, X):
    """A X for CSC A (plain loops over columns via numpy)."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X.reshape(-1, 1)
    cols = np.repeat(np.arange(n), np.diff(colptr))
    Y = np.zeros((n, X.shape[1]))
    np.add.at(Y, rowidx, values[:, None] * X[cols])
    return Y


def backward_error(n, colptr, rowidx, values, X, B):
    """Normwise backward error per right-hand side,
    ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf); returns the max."""
    X = np.asarray(X).reshape(n, -1)
    B = np.asarray(B).reshape(n, -1)
    R = B - matvec(n, colptr, rowidx, values, X)
    rs = np.zeros(n)
    np.add.at(rs, rowidx, np.abs(values))
    an = rs.max() if n else 0.0
    out = 0.0
    for c in range(X.shape[1]):
        den = an * np.abs(X[:, c]).max() + np.abs(B[:, c]).max()
        out = max(out, np.abs(R[:, c]).max() / den if den > 0 else 0.0)
    return out
