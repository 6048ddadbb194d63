"""The allocation-free refined solve, slu_solve_refine_noalloc, called through
the C ABI.

This entry point exists for callers that may not allocate device memory
when they solve (a device memory budget handed out entirely at start-up, a
framework that owns all device memory through its own pool, a loop that
cannot afford cudaMalloc's implicit synchronization).  It must give the
same answer as the allocating slu_solve, on two calls in a row (the second
call finds the first call's leftovers in the shared scratch array), and
must refuse problems larger than its fixed scratch.

The file name sorts last so that a run stopping at the first failure has
run every other test before this one."""
import ctypes as C

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
S = pytest.importorskip("paper_2512_04389_b300.slu")

TOL = 1e-10          # relative tolerance used by the solve parity tests
MAX_ELEMS = 1 << 20  # SLU_NOALLOC_MAX_ELEMS in include/slu.h


def _dev(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def _noalloc(F, B):
    Bc = B.t().contiguous().t()
    n, k = Bc.shape
    X = torch.empty((k, n), dtype=torch.float64, device="cuda").t()
    info = S.SolveInfo()
    st = S.lib.slu_solve_refine_noalloc(
        F._h, C.c_void_p(Bc.data_ptr()), n, k, C.c_void_p(X.data_ptr()), n,
        C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(info))
    return st, X, info


def _single(prec, nrhs):
    s = workloads.grid7_cd(14, nrhs=nrhs)
    P = S.Plan(s.n, s.colptr, s.rowidx, b_min=16, precision=prec)
    return P, _dev(s.values), _dev(s.rhs)


def _members(prec, nrhs):
    """A slu_analyze_batch plan: the backward error is taken per member."""
    ms = workloads.batch_grid5(count=8, seed=4, k_lo=16, k_hi=40)
    P = S.Plan([m.n for m in ms], [m.colptr for m in ms],
               [m.rowidx for m in ms], precision=prec)
    vals = np.concatenate([m.values for m in ms])
    rng = np.random.Generator(np.random.PCG64(7))
    # members' right-hand sides of very different scales, so that a batch-
    # wide norm would misjudge the small members' backward errors
    B = np.concatenate([rng.standard_normal((m.n, nrhs)) * 10.0 ** (3 * (q % 3))
                        for q, m in enumerate(ms)])
    return P, _dev(vals), _dev(B)


CASES = [("single", "fp32", 3), ("single", "fp64", 3),
         ("single", "fp32", 6),          # more than one 4-column sweep chunk
         ("batch", "fp32", 1), ("batch", "fp64", 2), ("batch", "fp32", 6)]


@pytest.mark.parametrize("kind,prec,nrhs", CASES,
                         ids=[f"{k}-{p}-{r}rhs" for k, p, r in CASES])
def test_noalloc_matches_allocating_solve_twice(kind, prec, nrhs):
    P, vals, B = (_single if kind == "single" else _members)(prec, nrhs)
    F = S.Factor(P, vals)
    Xref, iref = F.solve(B, info=True)
    Xref = Xref.cpu().numpy()
    for _ in range(2):
        st, X, info = _noalloc(F, B)
        assert st == 0, S.lib.slu_last_error().decode()
        Xg = X.cpu().numpy()
        assert np.abs(Xg - Xref).max() <= TOL * np.abs(Xref).max()
        assert info.iterations == iref["iterations"]
        assert info.backward_error <= (1e-14 if prec == "fp32" else 1e-13)
        assert info.backward_error == pytest.approx(iref["backward_error"],
                                                    rel=1e-12, abs=1e-300)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    s = workloads.grid5(130)                      # n = 16,900
    P = S.Plan(s.n, s.colptr, s.rowidx)
    F = S.Factor(P, _dev(s.values))
    nrhs = 64                                     # 16,900 * 64 > 2^20
    assert s.n * nrhs > MAX_ELEMS
    B = torch.ones((s.n, nrhs), dtype=torch.float64, device="cuda")
    st, _, _ = _noalloc(F, B)
    assert st == 1
    assert "SLU_NOALLOC_MAX_ELEMS" in S.lib.slu_last_error().decode()
    st, X, info = _noalloc(F, B[:, :2])           # within the limit: fine
    assert st == 0 and info.backward_error <= 1e-13
