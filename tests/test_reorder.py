"""General-matrix front end (slu_reorder, host): the maximum-product
transversal against scipy's dense assignment solver, the scaling's defining
property, recovery of a hidden row permutation, structural singularity, the
nested-dissection ordering's fill (counted by the oracle's LU) and the
reordered matrix against a dense computation."""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import workloads
from conftest import dense_to_csc
from oracle import lu as OL

S = pytest.importorskip("paper_2512_04389_b300.slu")


def _random_sparse(n, density, seed):
    rng = np.random.default_rng(seed)
    M = rng.random((n, n)) < density
    M[rng.permutation(n), np.arange(n)] = True          # a perfect matching exists
    A = np.where(M, rng.uniform(-1, 1, (n, n)) * 10.0 ** rng.uniform(-3, 3, (n, n)), 0.0)
    return A


@pytest.mark.parametrize("n,density,seed", [(12, 0.3, 1), (40, 0.15, 2), (60, 0.08, 3),
                                            (60, 0.5, 4)])
def test_matching_is_a_maximum_product_transversal(n, density, seed):
    A = _random_sparse(n, density, seed)
    cp, ri, vx = dense_to_csc(A)
    R = S.Reordering(n, cp, ri, vx, scale=True, order=False)
    got = np.sum(np.log(np.abs(A[R.rowperm, R.colperm])))
    cost = np.where(A != 0, -np.log(np.abs(np.where(A != 0, A, 1.0))), 1e6)
    r, c = linear_sum_assignment(cost)
    best = -cost[r, c].sum()
    assert np.all(A[R.rowperm, R.colperm] != 0)
    assert got == pytest.approx(best, abs=1e-9 * max(1.0, abs(best)))
    # scaled: matched entries of magnitude 1, none above 1
    Rm = R.rowscale[:, None] * A * R.colscale[None, :]
    assert np.allclose(np.abs(Rm[R.rowperm, R.colperm]), 1.0, rtol=1e-12)
    assert np.abs(Rm).max() <= 1.0 + 1e-12


def test_matching_recovers_a_hidden_row_permutation():
    """A diagonally dominant matrix with its rows shuffled: the largest-
    product transversal is the original diagonal."""
    s = workloads.grid5(20)
    A = s.dense()
    p = np.random.default_rng(5).permutation(s.n)
    B = A[p]                                             # row k of B = row p[k] of A
    cp, ri, vx = dense_to_csc(B)
    R = S.Reordering(s.n, cp, ri, vx, scale=True, order=False)
    # column j is matched to B's row holding A's diagonal entry (j, j)
    inv = np.argsort(p)
    assert np.array_equal(R.rowperm, inv[R.colperm])


@pytest.mark.parametrize("kind", ["empty_column", "deficient"])
def test_structurally_singular_is_reported(kind):
    A = np.eye(6)
    if kind == "empty_column":
        A[:, 2] = 0.0
    else:                     # columns 1 and 2 hold entries in row 1 only
        A[:, 1] = 0.0
        A[:, 2] = 0.0
        A[1, 1] = A[1, 2] = 1.0
        A[2, 2] = 0.0
        A[2, 0] = 1.0
        A[2, 3] = 1.0
        A[2, 2] = 0.0
    cp, ri, vx = dense_to_csc(A, A != 0)
    with pytest.raises(S.SluError) as ei:
        S.Reordering(6, cp, ri, vx)
    assert ei.value.status == 4


def _fill(n, cp, ri, vx):
    F = OL.lu(n, cp, ri, vx)
    return OL.lu_pattern(F)[1].size


def test_nested_dissection_reduces_fill_of_a_scrambled_grid():
    """A 40 x 40 grid in a random symmetric order: the ordering's fill
    (oracle LU) is within 1.6x the geometric nested dissection's and far
    below the scrambled order's."""
    s = workloads.grid5(40)
    A = s.dense()
    q = np.random.default_rng(6).permutation(s.n)
    B = A[np.ix_(q, q)]
    cp, ri, vx = dense_to_csc(B)
    R = S.Reordering(s.n, cp, ri, vx, scale=False, order=True, leaf=16)
    assert np.array_equal(np.sort(R.colperm), np.arange(s.n))
    assert np.array_equal(R.rowperm, R.colperm)          # no matching: symmetric
    rcp, rri, rvx = R.matrix()
    nd = _fill(s.n, rcp, rri, rvx)
    geo = _fill(s.n, s.colptr, s.rowidx, s.values)
    scr = _fill(s.n, cp, ri, vx)
    print(f"fill: ordering {nd}, geometric ND {geo}, scrambled {scr}")
    assert nd <= 1.6 * geo and nd <= 0.5 * scr


def test_reordered_matrix_equals_dense_computation():
    A = _random_sparse(30, 0.2, 7)
    cp, ri, vx = dense_to_csc(A)
    R = S.Reordering(30, cp, ri, vx, scale=True, order=True, leaf=4)
    rcp, rri, rvx = R.matrix()
    D = np.zeros((30, 30))
    for j in range(30):
        for q in range(rcp[j], rcp[j + 1]):
            D[rri[q], j] = rvx[q]
        assert np.all(np.diff(rri[rcp[j]:rcp[j + 1]]) > 0)      # rows sorted
    want = (R.rowscale[:, None] * A * R.colscale[None, :])[np.ix_(R.rowperm, R.colperm)]
    assert np.allclose(D, want, rtol=1e-15, atol=0)
    assert np.allclose(np.abs(np.diag(D)), 1.0, rtol=1e-12)


def test_reorder_rejects_bad_input():
    cp = np.array([0, 1, 2], np.int64)
    ri = np.array([0, 1], np.int32)
    with pytest.raises(S.SluError):
        S.Reordering(2, cp, ri, None, scale=True)          # scaling needs values
    with pytest.raises(S.SluError):
        S.Reordering(2, cp, ri, np.array([1.0, np.nan]))
