"""Host-side argument checks of the Python binding: a value vector or a
right-hand side of the wrong size is refused before any pointer reaches
the library (the kernels read exactly nnz(A) values and n rows)."""
import numpy as np
import pytest
import torch

import workloads

S = pytest.importorskip("paper_2512_04389_b300.slu")


@pytest.fixture(scope="module")
def plan():
    s = workloads.grid5(6)
    return S.Plan(s.n, s.colptr, s.rowidx)


@pytest.mark.parametrize("bad", ["short", "long", "matrix", "strided"])
def test_factor_rejects_misshapen_values(plan, bad):
    nnz = plan.info["nnz_a"]
    v = {"short": torch.zeros(nnz - 1, dtype=torch.float64),
         "long": torch.zeros(nnz + 1, dtype=torch.float64),
         "matrix": torch.zeros(1, nnz, dtype=torch.float64),
         "strided": torch.zeros(2 * nnz, dtype=torch.float64)[::2]}[bad]
    with pytest.raises(ValueError, match="values"):
        S.Factor(plan, v)


def test_factor_accepts_shape_then_requires_device(plan):
    v = torch.zeros(plan.info["nnz_a"], dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        S.Factor(plan, v)


def test_rows_check(plan):
    n = plan.n
    S._check_rows(torch.zeros(n), n, "B")
    S._check_rows(torch.zeros(n, 3), n, "B")
    S._check_rows(torch.zeros(n, 0), n, "B")
    for bad in (torch.zeros(n + 1), torch.zeros(n - 1, 2), torch.zeros(n, 2, 1),
                torch.zeros(())):
        with pytest.raises(ValueError, match="rows"):
            S._check_rows(bad, n, "B")


def test_empty_plan_values(plan):
    P0 = S.Plan(0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    with pytest.raises(ValueError, match="CUDA"):
        S.Factor(P0, torch.zeros(0, dtype=torch.float64))


@pytest.mark.parametrize("bad", ["short_colptr", "long_colptr", "short_rowidx",
                                 "negative_n", "matrix_colptr"])
def test_plan_rejects_short_pattern_arrays(bad):
    """The library reads colptr[0..n] and rowidx[0..colptr[n]) from host
    memory; arrays shorter than that are refused before the call."""
    s = workloads.grid5(5)
    n, cp, ri = s.n, s.colptr, s.rowidx
    if bad == "short_colptr":
        cp = cp[:-1]
    elif bad == "long_colptr":
        cp = np.append(cp, cp[-1])
    elif bad == "short_rowidx":
        ri = ri[:-1]
    elif bad == "negative_n":
        n = -1
    else:
        cp = cp[None, :]
    with pytest.raises(ValueError):
        S.Plan(n, cp, ri)


def test_plan_accepts_longer_rowidx_and_batch_lengths():
    s = workloads.grid5(5)
    P = S.Plan(s.n, s.colptr, np.append(s.rowidx, [0, 0]))
    assert P.info["nnz_a"] == s.nnz
    with pytest.raises(ValueError, match="orders"):
        S.Plan([s.n, s.n], [s.colptr], [s.rowidx, s.rowidx])
    with pytest.raises(ValueError):
        S.Plan([s.n, s.n], [s.colptr, s.colptr[:-1]], [s.rowidx, s.rowidx])
