"""Persistent solve (slu_set_persistent_solve): every sweep in one launch per
four right-hand sides, blocks started by device-side counters.  The
solutions must be bit for bit those of the per-level launches (the same
operations in the same order), for both storage precisions, the transposed
solve, several right-hand-side counts, batch plans and the refined FP32
solve; plans with a diagonal block that has no explicit inverse are
refused."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
S = pytest.importorskip("paper_2512_04389_b300.slu")


def _dev(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.float64, device="cuda")


CASES = [
    ("grid7cd_12", lambda: workloads.grid7_cd(12), {}),
    ("grid5_40", lambda: workloads.grid5(40), {"b_min": 8}),
    ("theta_12", lambda: workloads.grid7_theta(12), {"sample_points": 2000, "max_num": 1}),
    ("grid7cd_10 regular 24", lambda: workloads.grid7_cd(10), {"blocking": "regular",
                                                                "regular_block": 24}),
]


def _pair(s, prec, opts):
    P = S.Plan(s.n, s.colptr, s.rowidx, precision=prec, dense_threshold=0.0, **opts)
    F = S.Factor(P, _dev(s.values))
    return P, F


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,make,opts", CASES, ids=[c[0] for c in CASES])
def test_persistent_solve_equals_per_level_solve(name, make, opts, prec):
    s = make()
    _, F = _pair(s, prec, opts)
    rng = np.random.default_rng(3)
    for k in (1, 4, 6):
        B = _dev(rng.standard_normal((s.n, k)))
        F.set_persistent_solve(False)
        x0 = F.solve(B.clone()).cpu().numpy()
        t0 = F.solve_transpose(B.clone()).cpu().numpy()
        F.set_persistent_solve(True)
        x1 = F.solve(B.clone()).cpu().numpy()
        t1 = F.solve_transpose(B.clone()).cpu().numpy()
        assert np.array_equal(x0, x1), (name, prec, k)
        assert np.array_equal(t0, t1), (name, prec, k)


def test_persistent_solve_launches_once_per_sweep():
    s = workloads.grid7_cd(12)
    P, F = _pair(s, "fp64", {})
    F.set_persistent_solve(True)
    B = _dev(np.ones((s.n, 6)))
    F.solve(B)                                      # records the graph
    torch.cuda.synchronize()
    l0 = F.stats()["launches"]
    x = F.solve(B)
    torch.cuda.synchronize()
    # two sweeps, two chunks of at most 4 right-hand sides, one launch each
    assert F.stats()["launches"] - l0 == 4
    r = s.dense() @ x.cpu().numpy() - np.ones((s.n, 6))
    assert np.abs(r).max() < 1e-9


def test_persistent_refined_fp32_solve_equals_per_level():
    s = workloads.grid7_cd(14)
    _, F = _pair(s, "fp32", {})
    b = _dev(s.rhs)
    x0, i0 = F.solve(b, info=True)
    F.set_persistent_solve(True)
    x1, i1 = F.solve(b, info=True)
    assert np.array_equal(x0.cpu().numpy(), x1.cpu().numpy())
    assert i0 == i1 and i1["backward_error"] <= 1e-14


def test_persistent_solve_on_a_batch_plan():
    ms = workloads.batch_grid5(count=10, seed=9, k_lo=8, k_hi=30)
    PB = S.Plan([m.n for m in ms], [m.colptr for m in ms], [m.rowidx for m in ms],
                dense_threshold=0.0, b_min=8)
    F = S.Factor(PB, _dev(np.concatenate([m.values for m in ms])))
    B = _dev(np.concatenate([m.rhs for m in ms]))
    x0 = F.solve(B).cpu().numpy()
    F.set_persistent_solve(True)
    x1 = F.solve(B).cpu().numpy()
    assert np.array_equal(x0, x1)


def test_persistent_solve_needs_explicit_inverses():
    s = workloads.grid5(30)                         # two diagonal blocks of 450 rows
    P = S.Plan(s.n, s.colptr, s.rowidx, blocking="regular", regular_block=450)
    F = S.Factor(P, _dev(s.values))
    with pytest.raises(S.SluError) as e:
        F.set_persistent_solve(True)
    assert e.value.status == 7
    F.set_persistent_solve(False)                   # always allowed
