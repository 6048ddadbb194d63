"""Pins of the CPU oracle's LU, solves, flop count and backward error to
results fixed independently of the oracle: known factors, a library LU,
brute-force fill, closed forms."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from oracle import lu as OL
from conftest import brute_fill, random_sym_pattern, dense_to_csc


def _dense_factors(F):
    n = F["n"]
    L = np.eye(n)
    U = np.zeros((n, n))
    lc = np.repeat(np.arange(n), np.diff(F["Lp"]))
    uc = np.repeat(np.arange(n), np.diff(F["Up"]))
    L[F["Li"], lc] = F["Lx"]
    U[F["Ui"], uc] = F["Ux"]
    return L, U


@pytest.mark.parametrize("n,density", [(40, 0.05), (120, 0.02), (200, 0.01)])
def test_exact_recovery_of_known_factors(n, density, rng):
    """A = L0 U0 with L0 unit lower and U0 upper on a pattern closed under
    fill: the LU without row exchanges is unique, so the oracle must return
    L0 and U0 (up to rounding) and exactly their pattern."""
    F0 = brute_fill(random_sym_pattern(n, density, rng))
    L0 = np.where(np.tril(F0, -1), rng.uniform(-0.5, 0.5, (n, n)), 0.0)
    L0 /= np.maximum(1.0, np.sqrt(np.tril(F0, -1).sum(1, keepdims=True)))
    L0 += np.eye(n)
    U0 = np.where(np.triu(F0, 1), rng.uniform(-0.5, 0.5, (n, n)), 0.0)
    U0 /= np.maximum(1.0, np.sqrt(np.triu(F0, 1).sum(0, keepdims=True)))
    d = rng.uniform(1.0, 2.0, n) * np.where(rng.random(n) < 0.5, -1, 1)
    U0 += np.diag(d)
    A = L0 @ U0
    ap, ai, ax = dense_to_csc(A, F0)
    F = OL.lu(n, ap, ai, ax)
    L, U = _dense_factors(F)
    assert np.array_equal(_pattern_lower(F, n), np.tril(F0, -1))
    assert np.array_equal(_pattern_upper(F, n), np.triu(F0))
    scale = max(np.abs(L0).max(), np.abs(U0).max())
    assert np.abs(L - L0).max() / scale <= 1e-12
    assert np.abs(U - U0).max() / scale <= 1e-12


def _pattern_lower(F, n):
    P = np.zeros((n, n), bool)
    P[F["Li"], np.repeat(np.arange(n), np.diff(F["Lp"]))] = True
    return P


def _pattern_upper(F, n):
    P = np.zeros((n, n), bool)
    P[F["Ui"], np.repeat(np.arange(n), np.diff(F["Up"]))] = True
    return P


@pytest.mark.parametrize("n", [1, 2, 7, 33, 64])
def test_dense_matches_library_lu(n, rng):
    """On a column-diagonally-dominant dense matrix partial pivoting makes no
    row exchange, so LAPACK's GETRF (scipy.linalg.lu) is the no-pivot LU."""
    A = rng.uniform(-1, 1, (n, n))
    A += np.diag(np.abs(A).sum(0) + 0.5)
    P, Ll, Ul = sla.lu(A)
    assert np.array_equal(P, np.eye(n))
    ap, ai, ax = dense_to_csc(A, np.ones((n, n), bool))
    L, U = _dense_factors(OL.lu(n, ap, ai, ax))
    assert np.abs(L - Ll).max() <= 1e-13 * np.abs(Ll).max()
    assert np.abs(U - Ul).max() <= 1e-13 * np.abs(Ul).max()


@pytest.mark.parametrize("n,density", [(50, 0.04), (300, 0.006), (500, 0.004)])
def test_symbolic_fill_matches_boolean_elimination(n, density, rng):
    P = random_sym_pattern(n, density, rng)
    A = np.where(P, rng.uniform(-1, 1, (n, n)), 0.0)
    A += np.diag(np.abs(A).sum(1) + 1.0)
    ap, ai, ax = dense_to_csc(A, P)
    F = OL.lu(n, ap, ai, ax)
    fill = brute_fill(P)
    assert np.array_equal(_pattern_lower(F, n), np.tril(fill, -1))
    assert np.array_equal(_pattern_upper(F, n), np.triu(fill))


def test_symbolic_fill_grid_nd():
    s = workloads.grid5(12)
    P = s.dense() != 0
    P |= P.T
    F = OL.lu(s.n, s.colptr, s.rowidx, s.values)
    fill = brute_fill(P)
    assert np.array_equal(_pattern_lower(F, s.n), np.tril(fill, -1))
    assert np.array_equal(_pattern_upper(F, s.n), np.triu(fill))


def test_nonsymmetric_input_is_symmetrized():
    """An entry present only in A(i,j) makes (j,i) structural too."""
    A = np.array([[4.0, 1.0, 0.0], [0.0, 4.0, 0.0], [2.0, 0.0, 4.0]])
    ap, ai, ax = dense_to_csc(A)
    F = OL.lu(3, ap, ai, ax)
    L, U = _dense_factors(F)
    assert np.allclose(L @ U, A, atol=1e-15)
    assert _pattern_lower(F, 3)[1, 0] and _pattern_upper(F, 3)[0, 2]


def _residual(s):
    F = OL.lu(s.n, s.colptr, s.rowidx, s.values)
    L, U = _dense_factors(F)
    A = s.dense()
    return np.linalg.norm(A - L @ U) / np.linalg.norm(A)


@pytest.mark.parametrize("mk", [lambda: workloads.grid5(48),
                                lambda: workloads.grid7_theta(6),
                                lambda: workloads.grid7_cd(10),
                                lambda: workloads.circuit_bbd(
                                    n=1500, border=30, block_lo=20,
                                    block_hi=60)])
def test_residual_small_configs(mk):
    assert _residual(mk()) <= 1e-14


def test_solves_against_dense(rng):
    s = workloads.grid7_cd(6, nrhs=3)
    F = OL.lu(s.n, s.colptr, s.rowidx, s.values)
    A = s.dense()
    X = OL.solve(F, s.rhs)
    assert np.abs(X - np.linalg.solve(A, s.rhs)).max() <= 1e-12
    G = rng.standard_normal((s.n, 2))
    Lam = OL.solve_transpose(F, G)
    assert np.abs(Lam - np.linalg.solve(A.T, G)).max() <= 1e-12


def test_pivot_perturbation_closed_form():
    """[[0, 1], [1, 1]] has a zero first pivot.  With tau the pivot becomes
    +tau (sign of zero is +): U = [[tau, 1], [0, 1 - 1/tau]], L21 = 1/tau."""
    A = np.array([[0.0, 1.0], [1.0, 1.0]])
    ap, ai, ax = dense_to_csc(A, np.ones((2, 2), bool))
    with pytest.raises(OL.SingularError):
        OL.lu(2, ap, ai, ax, tau=0.0)
    tau = 1e-3
    F = OL.lu(2, ap, ai, ax, tau=tau)
    L, U = _dense_factors(F)
    assert F["nperturb"] == 1
    assert np.allclose(U, [[tau, 1.0], [0.0, 1.0 - 1.0 / tau]], rtol=1e-15)
    assert np.isclose(L[1, 0], 1.0 / tau, rtol=1e-15)
    # negative small pivot keeps its sign
    A2 = np.array([[-1e-9, 1.0], [1.0, 1.0]])
    ap, ai, ax = dense_to_csc(A2, np.ones((2, 2), bool))
    F = OL.lu(2, ap, ai, ax, tau=tau)
    assert F["Ux"][0] == -tau and F["nperturb"] == 1


def test_flops_closed_form_dense():
    """Dense n x n, no fill beyond full: l_k = u_k = n-1-k, so
    flops = sum_m (m + 2 m^2), m = 0..n-1."""
    n = 17
    A = np.ones((n, n)) + n * np.eye(n)
    ap, ai, ax = dense_to_csc(A)
    F = OL.lu(n, ap, ai, ax)
    m = np.arange(n)
    assert OL.flops(F) == int(np.sum(m + 2 * m * m))


def test_backward_error_closed_form():
    """A = 2 I, b = 1, x = 0.5 + d: r = -2 d, so the normwise backward error
    is 2|d| / (2 (0.5 + d) + 1)."""
    n = 5
    ap = np.arange(n + 1, dtype=np.int64)
    ai = np.arange(n, dtype=np.int32)
    ax = np.full(n, 2.0)
    d = 1e-3
    x = np.full(n, 0.5 + d)
    be = OL.backward_error(n, ap, ai, ax, x, np.ones(n))
    assert np.isclose(be, 2 * d / (2 * (0.5 + d) + 1), rtol=1e-12)
    assert OL.backward_error(n, ap, ai, ax, np.full(n, 0.5), np.ones(n)) == 0


def test_matvec_and_backward_error_nonsymmetric_closed_form():
    """A = [[4, -1, 0], [2, 5, 0], [0, 3, 1]]: row sums 5, 7, 4 (||A||_inf =
    7) differ from column sums 6, 9, 1, and A^T x differs from A x, so a
    transposed product or the wrong norm fails.  x1 = 1 gives A x1 = (3, 7,
    4); b1 = A x1 + (0, 0.01, 0) has residual 0.01 and backward error
    0.01 / (7 * 1 + 7.01).  x2 = (0, 2, 0), b2 = A x2 = (-2, 10, 6) exactly:
    backward error 0, so the max over both columns is column 1's."""
    A = np.array([[4.0, -1.0, 0.0], [2.0, 5.0, 0.0], [0.0, 3.0, 1.0]])
    ap, ai, ax = dense_to_csc(A)
    X = np.array([[1.0, 0.0], [1.0, 2.0], [1.0, 0.0]])
    Y = OL.matvec(3, ap, ai, ax, X)
    assert np.array_equal(Y, np.array([[3.0, -2.0], [7.0, 10.0], [4.0, 6.0]]))
    B = Y.copy()
    B[1, 0] += 0.01
    be = OL.backward_error(3, ap, ai, ax, X, B)
    assert np.isclose(be, 0.01 / (7.0 + 7.01), rtol=1e-12)
    assert OL.backward_error(3, ap, ai, ax, X[:, 1], B[:, 1]) == 0.0


def test_generator_shapes_match_named_configs():
    assert workloads.grid5(48).nnz == 11_328
    assert workloads.grid7_theta(32).nnz == 223_232
    s = workloads.grid7_cd(8)
    A = s.dense()
    off = A - np.diag(np.diag(A))
    assert np.all(np.diag(A) > np.abs(off).sum(1))      # strict row dominance
