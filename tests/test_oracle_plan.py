"""Pins of the oracle's blocking and block plan: closed forms of the diagonal
block pointer (Section 4.2), hand-derived irregular blockings (Section 4.3,
Algorithm 3), brute-force longest chains of the explicit task graph of
Algorithm 1, and a numpy execution of the plan's tasks that must reproduce
the oracle's factors."""
import numpy as np
import pytest

import workloads
from oracle import lu as OL, plan as OP
from conftest import random_sym_pattern, dense_to_csc, brute_fill


def _brute_bp(P):
    n = P.shape[0]
    return np.array([P[:k, :k].sum() for k in range(n + 1)], dtype=np.int64)


@pytest.mark.parametrize("n,density", [(1, 1.0), (9, 0.3), (60, 0.05)])
def test_blockptr_brute_force(n, density, rng):
    P = random_sym_pattern(n, density, rng)
    ap, ai, _ = dense_to_csc(P.astype(float), P)
    assert np.array_equal(OP.blockptr(n, ap, ai), _brute_bp(P))


def test_blockptr_closed_forms():
    """Tridiagonal: bp[k] = 3k - 2 (k >= 1), a linear curve; dense: k^2, a
    quadratic curve (Section 4.2); arrowhead (diagonal plus last row and
    column): bp[k] = k for k < n and 3n - 2 at n, a jump at the end."""
    n = 50
    k = np.arange(n + 1)
    T = np.eye(n, dtype=bool) | np.eye(n, k=1, dtype=bool) | \
        np.eye(n, k=-1, dtype=bool)
    ap, ai, _ = dense_to_csc(T.astype(float), T)
    assert np.array_equal(OP.blockptr(n, ap, ai), np.where(k > 0, 3 * k - 2, 0))
    D = np.ones((n, n), bool)
    ap, ai, _ = dense_to_csc(D.astype(float), D)
    assert np.array_equal(OP.blockptr(n, ap, ai), k * k)
    Ar = np.eye(n, dtype=bool)
    Ar[-1, :] = Ar[:, -1] = True
    ap, ai, _ = dense_to_csc(Ar.astype(float), Ar)
    exp = k.copy()
    exp[n] = 3 * n - 2
    assert np.array_equal(OP.blockptr(n, ap, ai), exp)


N = 3200   # S = min(1000, 3200 // 32) = 100 samples, 32 rows apart


def test_irregular_tridiagonal_linear_profile():
    """bp = 3k - 2: window 0 gains 3*64 - 2 < 2/S of the total (bp[0] = 0),
    every later window gains 192 and 192 * 100 >= 2 * 9598: so one skip,
    then a boundary at every sample from idx(3)."""
    k = np.arange(N + 1)
    ptr = OP.irregular_ptr(np.where(k > 0, 3 * k - 2, 0), N)
    assert np.array_equal(ptr, np.r_[0, np.arange(3, 101) * 32])


def test_irregular_dense_quadratic_profile():
    """bp = k^2: window i gains (4i + 4)/S^2 of the total, dense iff
    i >= S/2 - 1 = 49 (equality at 49 exercises '>=').  Before that, runs of
    three skips then a forced boundary: idx(5), idx(9), ..., idx(49); one
    skip at i = 48; then a boundary at every sample from idx(51)."""
    k = np.arange(N + 1)
    ptr = OP.irregular_ptr(k * k, N)
    exp = np.r_[0, np.arange(5, 50, 4), np.arange(51, 101)] * 32
    assert np.array_equal(ptr, exp)


def test_irregular_dense_profile_stride_two():
    """Same curve, windows every 'step' samples: boundaries every 8 samples
    up to 48, a skip at i = 48, then dense windows every 2 from idx(52)."""
    k = np.arange(N + 1)
    ptr = OP.irregular_ptr(k * k, N, stride=2)
    exp = np.r_[0, np.arange(8, 49, 8), np.arange(52, 101, 2)] * 32
    assert np.array_equal(ptr, exp)


def test_irregular_arrowhead_jump():
    """bp = k with a jump to 3N - 2 at N: every window is sparse except the
    last one, so blocks of four samples (the first of five) and the final
    dense window [98, 100] closes at N."""
    k = np.arange(N + 1)
    bp = k.copy()
    bp[N] = 3 * N - 2
    ptr = OP.irregular_ptr(bp, N)
    exp = np.r_[0, np.arange(5, 98, 4), 100] * 32
    assert np.array_equal(ptr, exp)


def test_irregular_small_matrix_and_sampling():
    """S = min(1000, N // b_min); idx(s) = floor(s N / S)."""
    assert OP.num_samples(2304) == 72 and OP.num_samples(64_000) == 1000
    assert OP.num_samples(10) == 1
    assert np.array_equal(OP.sample_rows(10, 3), [0, 3, 6, 10])
    ptr = OP.irregular_ptr(np.arange(11) ** 2, 10)
    assert ptr[0] == 0 and ptr[-1] == 10 and np.all(np.diff(ptr) > 0)


def test_regular_ptr():
    assert np.array_equal(OP.regular_ptr(10, 4), [0, 4, 8, 10])
    assert np.array_equal(OP.regular_ptr(8, 4), [0, 4, 8])


def _pattern(s):
    F = OL.lu(s.n, s.colptr, s.rowidx, s.values)
    pp, pr, pv = OL.lu_pattern(F)
    return F, pp, pr


def _brute_levels(n, pp, pr, ptr):
    """Enumerate every task of Algorithm 1 (loops over all i, j, k) whose
    blocks are non-empty; step I' precedes step I when one of its tasks
    writes a block of block-row or block-column I.  Level = longest chain."""
    p = len(ptr) - 1
    cols = np.repeat(np.arange(n), np.diff(pp))
    bi = np.searchsorted(ptr, pr, side="right") - 1
    bj = np.searchsorted(ptr, cols, side="right") - 1
    NE = np.zeros((p, p), bool)
    NE[bi, bj] = True
    writes = {}
    for i in range(p):
        w = {(i, i)}
        for j in range(i + 1, p):
            if NE[i, j]:
                w.add((i, j))
            if NE[j, i]:
                w.add((j, i))
        for j in range(i + 1, p):
            for k in range(i + 1, p):
                if NE[k, i] and NE[i, j] and NE[k, j]:
                    w.add((k, j))
        writes[i] = w
    lev = np.zeros(p, dtype=np.int64)
    for I in range(p):
        best = -1
        for I2 in range(I):
            if any(a == I or b == I for (a, b) in writes[I2]):
                best = max(best, lev[I2])
        lev[I] = best + 1
    return lev


@pytest.mark.parametrize("mk,blocking", [
    (lambda: workloads.grid5(16), "irregular"),
    (lambda: workloads.grid5(16), 24),
    (lambda: workloads.grid7_theta(6), "irregular"),
    (lambda: workloads.circuit_bbd(n=900, border=20, block_lo=16,
                                   block_hi=48), "irregular")])
def test_levels_brute_force(mk, blocking):
    s = mk()
    _, pp, pr = _pattern(s)
    if blocking == "irregular":
        ptr = OP.irregular_ptr(OP.blockptr(s.n, pp, pr), s.n, b_min=8)
    else:
        ptr = OP.regular_ptr(s.n, blocking)
    plan = OP.block_plan(s.n, pp, pr, ptr)
    assert np.array_equal(plan["level"], _brute_levels(s.n, pp, pr, ptr))


def _lu_nopiv(B):
    B = B.copy()
    m = B.shape[0]
    for k in range(m):
        B[k + 1:, k] /= B[k, k]
        B[k + 1:, k + 1:] -= np.outer(B[k + 1:, k], B[k, k + 1:])
    return B


@pytest.mark.parametrize("mk", [lambda: workloads.grid5(20),
                                lambda: workloads.grid7_cd(7, nrhs=1)])
def test_plan_tasks_execute_to_oracle_factors(mk):
    """Run the plan's task lists level by level on dense numpy blocks (GETRF,
    GESSM, TSTRF, SSSSM of Algorithm 1) and compare with the oracle's L+U:
    a missing, duplicated or misplaced task changes the values."""
    s = mk()
    F, pp, pr = _pattern(s)
    ptr = OP.irregular_ptr(OP.blockptr(s.n, pp, pr), s.n, b_min=8)
    plan = OP.block_plan(s.n, pp, pr, ptr)
    A = s.dense()
    sl = [slice(ptr[i], ptr[i + 1]) for i in range(plan["p"])]
    B = A.copy()
    import scipy.linalg as sla
    for lv in range(plan["nlevels"]):
        for I in plan["getrf"][lv]:
            B[sl[I], sl[I]] = _lu_nopiv(B[sl[I], sl[I]])
        for I, J in plan["gessm"][lv]:
            B[sl[I], sl[J]] = sla.solve_triangular(
                B[sl[I], sl[I]], B[sl[I], sl[J]], lower=True,
                unit_diagonal=True)
        for J, I in plan["tstrf"][lv]:
            B[sl[J], sl[I]] = sla.solve_triangular(
                B[sl[I], sl[I]], B[sl[J], sl[I]].T, trans="T",
                lower=False).T
        for (K, J), srcs in plan["ssssm"][lv]:
            for I in srcs:
                B[sl[K], sl[J]] -= B[sl[K], sl[I]] @ B[sl[I], sl[J]]
    Lo, Uo = np.eye(s.n), np.zeros((s.n, s.n))
    lc = np.repeat(np.arange(s.n), np.diff(F["Lp"]))
    uc = np.repeat(np.arange(s.n), np.diff(F["Up"]))
    Lo[F["Li"], lc] = F["Lx"]
    Uo[F["Ui"], uc] = F["Ux"]
    ref = np.tril(Lo, -1) + Uo
    assert np.abs(B - ref).max() <= 1e-12 * np.abs(ref).max()


def test_fill_of_generated_configs_matches_brute_force():
    s = workloads.grid7_theta(6)
    _, pp, pr = _pattern(s)
    P = s.dense() != 0
    fill = brute_fill(P | P.T)
    cols = np.repeat(np.arange(s.n), np.diff(pp))
    Q = np.zeros_like(fill)
    Q[pr, cols] = True
    assert np.array_equal(Q, fill)
