"""Batching form: many independent matrices factored level by level in the
same launches (block-diagonal batch plan), optionally replayed from a CUDA
graph; results must equal the per-matrix launch loop's."""
import numpy as np
import pytest

import workloads
from oracle import lu as OL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
S = pytest.importorskip("paper_2512_04389_b300.slu")


def _dev(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def _batch(count=12, seed=5):
    return workloads.batch_grid5(count=count, seed=seed, k_lo=16, k_hi=40)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_factors_equal_member_factors(prec):
    ms = _batch()
    PB = S.Plan([m.n for m in ms], [m.colptr for m in ms],
                [m.rowidx for m in ms], precision=prec)
    vals = np.concatenate([m.values for m in ms])
    FB = S.Factor(PB, _dev(vals))
    gb = FB.export_factors().cpu().numpy()
    eb = PB.export()
    pos = 0
    for m in ms:
        P = S.Plan(m.n, m.colptr, m.rowidx, precision=prec)
        F = S.Factor(P, _dev(m.values))
        g = F.export_factors().cpu().numpy()
        assert np.array_equal(gb[pos:pos + g.size], g)
        if prec == "fp64":
            Fo = OL.lu(m.n, m.colptr, m.rowidx, m.values)
            _, _, pv = OL.lu_pattern(Fo)
            assert np.abs(g - pv).max() <= 1e-10 * np.abs(pv).max()
        pos += g.size
    assert pos == gb.size == eb["rowidx"].size


def test_batch_fp32_refinement_per_member():
    ms = _batch(count=16, seed=9)
    PB = S.Plan([m.n for m in ms], [m.colptr for m in ms],
                [m.rowidx for m in ms], precision="fp32")
    FB = S.Factor(PB, _dev(np.concatenate([m.values for m in ms])))
    B = np.concatenate([m.rhs[:, 0] for m in ms])
    X, info = FB.solve(_dev(B), info=True)
    assert info["converged"] and info["backward_error"] <= 1e-14
    Xh = X.cpu().numpy()
    pos = 0
    for m in ms:
        be = OL.backward_error(m.n, m.colptr, m.rowidx, m.values,
                               Xh[pos:pos + m.n], m.rhs[:, 0])
        assert be <= 1e-14
        pos += m.n


def test_graph_replay_matches_plain_refactor():
    ms = _batch(count=8, seed=2)
    PB = S.Plan([m.n for m in ms], [m.colptr for m in ms],
                [m.rowidx for m in ms])
    v = _dev(np.concatenate([m.values for m in ms]))
    F = S.Factor(PB, v)
    ref = F.export_factors().clone()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        F.set_graph(True)
        v2 = v * 1.25
        F.refactor(v2)          # records
        F.refactor(v2)          # replays
        torch.cuda.current_stream().synchronize()
        F.set_graph(False)
    F2 = S.Factor(PB, v2)
    assert torch.equal(F.export_factors(), F2.export_factors())
    F.refactor(v)
    assert torch.equal(F.export_factors(), ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_factor_batch_of_independent_plans(prec):
    """slu_factor_batch over independent plans: every member's factors equal
    slu_factor's for its own plan bit for bit (FP64 also within 1e-10 of
    the oracle), its solves equal the separate handle's, a refactor of one
    member with new values equals a fresh factorization, and the members
    can be released in any order."""
    ms = _batch(count=10, seed=21)
    plans = [S.Plan(m.n, m.colptr, m.rowidx, precision=prec) for m in ms]
    vals = [_dev(m.values) for m in ms]
    members = S.factor_batch(plans, vals)
    assert len(members) == len(ms)
    for q, (m, P, Fm) in enumerate(zip(ms, plans, members)):
        F = S.Factor(P, vals[q])
        g = Fm.export_factors()
        assert torch.equal(g, F.export_factors())
        if prec == "fp64":
            Fo = OL.lu(m.n, m.colptr, m.rowidx, m.values)
            _, _, pv = OL.lu_pattern(Fo)
            assert np.abs(g.cpu().numpy() - pv).max() <= 1e-10 * np.abs(pv).max()
        B = _dev(m.rhs[:, :1])
        X1, i1 = Fm.solve(B, info=True)
        X2, i2 = F.solve(B, info=True)
        assert torch.equal(X1, X2) and i1 == i2
        assert i1["backward_error"] <= (1e-13 if prec == "fp64" else 1e-14)
    q = 3
    v2 = vals[q] * 2.0
    members[q].refactor(v2, sync_info=True)
    F2 = S.Factor(plans[q], v2)
    assert torch.equal(members[q].export_factors(), F2.export_factors())
    order = np.random.default_rng(0).permutation(len(members))
    for q in order:                     # the shared factors go with the last
        members[q] = None


def test_factor_batch_rejects_mixed_options():
    ms = _batch(count=2, seed=22)
    plans = [S.Plan(ms[0].n, ms[0].colptr, ms[0].rowidx, precision="fp64"),
             S.Plan(ms[1].n, ms[1].colptr, ms[1].rowidx, precision="fp32")]
    with pytest.raises(S.SluError) as ei:
        S.factor_batch(plans, [_dev(m.values) for m in ms])
    assert ei.value.status == 7


def _dense_batch_plan(prec, count=12, seed=31, **kw):
    ms = _batch(count=count, seed=seed)
    P = S.Plan([m.n for m in ms], [m.colptr for m in ms],
               [m.rowidx for m in ms], precision=prec, dense_threshold=0.0, **kw)
    return ms, P, _dev(np.concatenate([m.values for m in ms]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["batch", "single"])
def test_persistent_launch_equals_per_level_launches(prec, kind):
    """One persistent launch for the level walk gives the per-level
    launches' factors bit for bit (batch plan and a single matrix), also
    replayed from a CUDA graph; the walk is a single kernel launch after
    the value scatter, and solves work on its factors."""
    if kind == "batch":
        _, P, v = _dense_batch_plan(prec)
    else:
        s = workloads.grid7_cd(14, nrhs=1)
        P = S.Plan(s.n, s.colptr, s.rowidx, precision=prec, dense_threshold=0.0,
                   b_min=16)
        v = _dev(s.values)
    P.check()
    F = S.Factor(P, v)
    ref = F.export_factors()
    F.set_persistent(True)
    l0 = F.stats()["launches"]
    F.refactor(v, sync_info=True)
    assert F.stats()["launches"] - l0 <= 5   # prep (3, 4 for a batch) + the walk (1)
    assert torch.equal(F.export_factors(), ref)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        F.set_graph(True)
        for _ in range(2):                          # record, then replay
            F.refactor(v)
        F.set_graph(False)
    torch.cuda.synchronize()
    assert torch.equal(F.export_factors(), ref)
    b = torch.ones(P.n, dtype=torch.float64, device="cuda")
    _, info = F.solve(b, info=True)
    assert info["converged"] and info["backward_error"] <= (
        1e-13 if prec == "fp64" else 1e-14)
    F.set_persistent(False)
    F.refactor(v, sync_info=True)
    assert torch.equal(F.export_factors(), ref)


def test_persistent_launch_needs_dense_blocks():
    s = workloads.grid5(24)
    P = S.Plan(s.n, s.colptr, s.rowidx, dense_threshold=2.0, b_min=8)
    F = S.Factor(P, _dev(s.values))
    with pytest.raises(S.SluError) as ei:
        F.set_persistent(True)
    assert ei.value.status == 7


def test_persistent_wait_that_cannot_be_met_times_out():
    """A work list whose dependency count can never be reached (set on the
    host) makes the bounded device-side waits run out: SLU_ERR_TIMEOUT (6)
    within the budget, the context stays usable, and with the list
    restored the factors are right again."""
    _, P, v = _dense_batch_plan("fp64", count=6, seed=33, wait_budget_ms=200)
    F = S.Factor(P, v)
    ref = F.export_factors()
    F.set_persistent(True)
    tasks = F.persistent_tasks()
    assert tasks.shape[0] > 0 and (tasks[:, 2] >= 0).any()
    bad = tasks.copy()
    t = int(np.nonzero(bad[:, 2] >= 0)[0][len(bad) // 3 % max(1, (bad[:, 2] >= 0).sum())])
    bad[t, 3] = 1 << 30                              # a count nothing reaches
    F.set_persistent_tasks(bad)
    with pytest.raises(S.SluError) as ei:
        F.refactor(v, sync_info=True)
    assert ei.value.status == 6 and "wait_budget_ms" in str(ei.value)
    F.set_persistent_tasks(tasks)
    F.refactor(v, sync_info=True)
    assert torch.equal(F.export_factors(), ref)
    with pytest.raises(S.SluError):                  # out-of-range entries refused
        bad2 = tasks.copy()
        bad2[0, 6] = 1 << 30
        F.set_persistent_tasks(bad2)
