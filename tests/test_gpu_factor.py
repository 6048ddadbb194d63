"""GPU parity: the library's factors and solves against the CPU oracle on the
same seeded inputs, through the C ABI.

Tolerances (FP64 path): max|dL, dU| / max|L, U| <= 1e-10 and solve backward
error <= 1e-13; FP32 factors refined in FP64 must reach backward error
<= 1e-14 (their factor error against the oracle is reported, not bounded
beyond what refinement needs)."""
import numpy as np
import pytest

import workloads
from oracle import lu as OL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
S = pytest.importorskip("paper_2512_04389_b300.slu")

FP64_TOL = 1e-10


def _dev(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def gpu_factor(s, **opts):
    P = S.Plan(s.n, s.colptr, s.rowidx, **opts)
    P.check()                  # every index the kernels read is in range
    F = S.Factor(P, _dev(s.values))
    return P, F


def oracle_factor(s):
    F = OL.lu(s.n, s.colptr, s.rowidx, s.values)
    pp, pr, pv = OL.lu_pattern(F)
    return F, pp, pr, pv


def factor_error(P, F, pv):
    got = F.export_factors().cpu().numpy()
    return np.abs(got - pv).max() / np.abs(pv).max()


CASES = [
    ("grid5_48", lambda: workloads.grid5(48), {}),
    ("grid5_48 regular64", lambda: workloads.grid5(48),
     dict(blocking="regular", regular_block=64)),
    ("grid5_48 stride2", lambda: workloads.grid5(48), dict(stride=2)),
    ("grid5_48 all dense", lambda: workloads.grid5(48),
     dict(dense_threshold=0.0)),
    ("grid5_48 all sparse", lambda: workloads.grid5(48),
     dict(dense_threshold=2.0)),
    ("grid7cd_14", lambda: workloads.grid7_cd(14, nrhs=4), dict(b_min=16)),
    ("grid7theta_12", lambda: workloads.grid7_theta(12), dict(b_min=16)),
    ("circuit_4000", lambda: workloads.circuit_bbd(
        n=4000, border=80, block_lo=16, block_hi=64), dict(b_min=16)),
    ("grid5_7 ragged", lambda: workloads.grid5(7), dict(b_min=3)),
    ("grid5_30 regular37", lambda: workloads.grid5(30),
     dict(blocking="regular", regular_block=37)),
    ("grid5_48 regular400 all dense", lambda: workloads.grid5(48),
     dict(blocking="regular", regular_block=400, dense_threshold=0.0)),
]


@pytest.mark.parametrize("name,mk,opts", CASES, ids=[c[0] for c in CASES])
def test_fp64_factor_and_solve_parity(name, mk, opts):
    s = mk()
    P, F = gpu_factor(s, **opts)
    Fo, pp, pr, pv = oracle_factor(s)
    e = P.export()
    assert np.array_equal(e["colptr"], pp) and np.array_equal(e["rowidx"], pr)
    assert factor_error(P, F, pv) <= FP64_TOL
    assert F.nperturb == 0
    X, info = F.solve(_dev(s.rhs), info=True)
    Xo = OL.solve(Fo, s.rhs)
    Xg = X.cpu().numpy()
    assert np.abs(Xg - Xo).max() / np.abs(Xo).max() <= 1e-10
    be = OL.backward_error(s.n, s.colptr, s.rowidx, s.values, Xg, s.rhs)
    assert be <= 1e-13
    assert abs(info["backward_error"] - be) <= 1e-15 + 0.01 * be
    G = np.random.default_rng(1).standard_normal((s.n, 2))
    Lam = F.solve_transpose(_dev(G)).cpu().numpy()
    Lo = OL.solve_transpose(Fo, G)
    assert np.abs(Lam - Lo).max() / np.abs(Lo).max() <= 1e-10


FP32_CASES = CASES[:1] + CASES[5:8] + CASES[-1:] + [
    ("circuit_20k", lambda: workloads.circuit_bbd(n=20_000, border=400),
     dict(dense_threshold=0.0)),
    ("grid7cd_14 all dense", lambda: workloads.grid7_cd(14, nrhs=4),
     dict(b_min=16, dense_threshold=0.0)),
    ("circuit_20k dense border", lambda: workloads.circuit_bbd(n=20_000, border=400),
     dict(dense_threshold=0.1))]


@pytest.mark.parametrize("name,mk,opts", FP32_CASES,
                         ids=[c[0] for c in FP32_CASES])
def test_fp32_factor_with_fp64_refinement(name, mk, opts):
    s = mk()
    P, F = gpu_factor(s, precision="fp32", **opts)
    _, _, _, pv = oracle_factor(s)
    err = factor_error(P, F, pv)
    assert err <= 1e-4          # reported; single-precision factors
    X, info = F.solve(_dev(s.rhs), info=True)
    be = OL.backward_error(s.n, s.colptr, s.rowidx, s.values,
                           X.cpu().numpy(), s.rhs)
    assert info["converged"] and info["backward_error"] <= 1e-14
    assert be <= 1e-14
    assert 1 <= info["iterations"] <= 10


def test_deterministic_and_refactor_identical():
    s = workloads.grid7_cd(12, nrhs=1)
    P, F = gpu_factor(s, b_min=16)
    a = F.export_factors().cpu().numpy()
    F2 = S.Factor(P, _dev(s.values))
    b = F2.export_factors().cpu().numpy()
    assert np.array_equal(a, b)
    v2 = s.values * 1.5
    F.refactor(_dev(v2))
    F.refactor(_dev(s.values))
    c = F.export_factors().cpu().numpy()
    assert np.array_equal(a, c)


def test_refactor_new_values_match_oracle():
    s = workloads.grid5(40)
    P, F = gpu_factor(s)
    rng = np.random.default_rng(7)
    v2 = s.values * rng.uniform(0.5, 1.5, s.values.size)
    F.refactor(_dev(v2))
    Fo = OL.lu(s.n, s.colptr, s.rowidx, v2)
    _, _, pv = OL.lu_pattern(Fo)
    assert factor_error(P, F, pv) <= FP64_TOL


def test_pivot_perturbation_and_singular():
    """A zero leading pivot: with perturbation the pivot becomes +tau
    (tau = 2^-26 max|A|) and is counted; without it the factor reports
    SINGULAR."""
    A = np.array([[0.0, 1.0, 0.0], [1.0, 1.0, 1.0], [0.0, 1.0, 3.0]])
    from conftest import dense_to_csc
    cp, ri, v = dense_to_csc(A, np.ones((3, 3), bool))
    P = S.Plan(3, cp, ri, b_min=1)
    F = S.Factor(P, _dev(v))
    assert F.nperturb == 1
    tau = 2.0 ** -26 * 3.0
    assert F.tau == pytest.approx(tau)
    Fo = OL.lu(3, cp, ri, v, tau=tau)
    _, _, pv = OL.lu_pattern(Fo)
    got = F.export_factors().cpu().numpy()
    assert np.abs(got - pv).max() / np.abs(pv).max() <= 1e-12
    P2 = S.Plan(3, cp, ri, b_min=1, pivot_perturb=0)
    with pytest.raises(S.SluError) as e:
        S.Factor(P2, _dev(v))
    assert e.value.status == 4


def test_empty_rhs_and_vector_rhs():
    s = workloads.grid5(16)
    P, F = gpu_factor(s, b_min=8)
    x = F.solve(_dev(s.rhs[:, 0]))
    assert x.shape == (s.n,)
    Fo = OL.lu(s.n, s.colptr, s.rowidx, s.values)
    xo = OL.solve(Fo, s.rhs[:, :1])[:, 0]
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-12 * np.abs(xo).max()


@pytest.mark.parametrize("name,mk,thr", [
    ("grid5_48 (2304)", lambda: workloads.grid5(48), 0.6),
    ("grid7theta_32 (32768)", lambda: workloads.grid7_theta(32), 0.6),
    ("grid7theta_32 all dense", lambda: workloads.grid7_theta(32), 0.0),
    ("circuit_20k (400 border)", lambda: workloads.circuit_bbd(
        n=20_000, border=400), 0.6),
    ("circuit_20k all dense", lambda: workloads.circuit_bbd(
        n=20_000, border=400), 0.0),
    ("circuit_20k dense border, sparse body", lambda: workloads.circuit_bbd(
        n=20_000, border=400), 0.1),
])
def test_full_size_parity(name, mk, thr):
    """Configurations the oracle factors in seconds: element-wise."""
    s = mk()
    P, F = gpu_factor(s, dense_threshold=thr)
    _, _, _, pv = oracle_factor(s)
    assert factor_error(P, F, pv) <= FP64_TOL
    X, info = F.solve(_dev(s.rhs), info=True)
    assert info["backward_error"] <= 1e-13


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tall_sparse_diagonal_blocks(prec):
    """Circuit matrix with blocks up to 512 rows (b_min 128): sparse
    diagonal blocks with dense border panels take the per-lane substitution
    with fewer than 32 vectors per warp (FP64: 16 for 512 rows)."""
    s = workloads.circuit_bbd(n=20_000, border=400)
    P, F = gpu_factor(s, b_min=128, dense_threshold=0.1, precision=prec)
    assert P.info["max_block"] > 450
    _, _, _, pv = oracle_factor(s)
    if prec == "fp64":
        assert factor_error(P, F, pv) <= FP64_TOL
    else:
        assert factor_error(P, F, pv) <= 1e-4
    X, info = F.solve(_dev(s.rhs), info=True)
    assert info["backward_error"] <= (1e-13 if prec == "fp64" else 1e-14)
    if prec == "fp32":
        assert info["iterations"] <= 3


def test_full_size_grid7cd_40_properties():
    """40^3 convection-diffusion (n = 64,000) in the benchmark's
    configuration: backward error of the solve, and A = L U checked on 2000
    sampled entries of A, each recomputed in FP64 from the exported factors."""
    s = workloads.grid7_cd(40)
    P, F = gpu_factor(s)
    X, info = F.solve(_dev(s.rhs), info=True)
    be = OL.backward_error(s.n, s.colptr, s.rowidx, s.values,
                           X.cpu().numpy(), s.rhs)
    assert be <= 1e-13
    e = P.export()
    vals = F.export_factors().cpu().numpy()
    cp, ri = e["colptr"], e["rowidx"]
    rng = np.random.default_rng(3)
    cols = np.repeat(np.arange(s.n), np.diff(s.colptr))
    pick = rng.choice(s.values.size, 2000, replace=False)
    # L(i, :) by rows: gather strictly-lower entries by row once
    lower = ri > np.repeat(np.arange(s.n), np.diff(cp))
    lr = ri[lower]
    lc = np.repeat(np.arange(s.n), np.diff(cp))[lower]
    lv = vals[lower]
    order = np.argsort(lr, kind="stable")
    lr, lc, lv = lr[order], lc[order], lv[order]
    lptr = np.searchsorted(lr, np.arange(s.n + 1))
    scale = np.abs(s.values).max()
    worst = 0.0
    for q in pick:
        i, j = s.rowidx[q], cols[q]
        ucol_r = ri[cp[j]:cp[j + 1]]
        ucol_v = vals[cp[j]:cp[j + 1]]
        um = ucol_r <= j
        u = dict(zip(ucol_r[um].tolist(), ucol_v[um].tolist()))
        acc = u.get(i, 0.0) if i <= j else 0.0          # L(i,i) = 1
        for k, lik in zip(lc[lptr[i]:lptr[i + 1]], lv[lptr[i]:lptr[i + 1]]):
            if k <= j and k in u:
                acc += lik * u[k]
        worst = max(worst, abs(acc - s.values[q]) / scale)
    assert worst <= 1e-12


def test_solve_graph_replay_matches_direct_launches():
    """Solves replay a recorded graph of the level sweeps; with profiling on
    the same sweeps run as direct launches.  Both give identical results,
    for several right-hand-side counts and the transposed solve."""
    s = workloads.grid7_cd(14, nrhs=6)
    P, F = gpu_factor(s, b_min=16, dense_threshold=0.0)
    B = _dev(s.rhs)
    for k in (1, 4, 6):
        x1 = F.solve(B[:, :k].contiguous())
        x2 = F.solve(B[:, :k].contiguous())          # replay
        F.set_profiling(True)
        x3 = F.solve(B[:, :k].contiguous())          # direct launches
        F.set_profiling(False)
        assert torch.equal(x1, x2) and torch.equal(x1, x3)
    t1 = F.solve_transpose(B)
    F.set_profiling(True)
    t2 = F.solve_transpose(B)
    F.set_profiling(False)
    assert torch.equal(t1, t2)


def test_autotuner_picks_a_candidate_and_caches(tmp_path, monkeypatch):
    from paper_2512_04389_b300 import tune as T
    monkeypatch.setenv("SLU_TUNE_CACHE", str(tmp_path / "tune.json"))
    s = workloads.grid5(32)
    best, timings = T.tune(s.n, s.colptr, s.rowidx, _dev(s.values),
                           _dev(s.rhs), precision="fp32")
    cands = T.default_candidates(s.n, {"precision": "fp32"})
    base = {k: v for k, v in best.items() if k != "tc_passes"}
    assert base in cands and best.get("tc_passes", 3) in T.TC_MODES
    # every blocking candidate, then the other tile modes of the best one
    assert len(timings) == len(cands) + len(T.TC_MODES) - 1
    again, t2 = T.tune(s.n, s.colptr, s.rowidx, _dev(s.values), _dev(s.rhs),
                       precision="fp32")
    assert again == best and t2 == timings          # served from the cache


# --- the benchmarked 40^3 configuration, with every option set the
# autotuner may pick for it (so the plan the benchmark times is among them)

@pytest.fixture(scope="module")
def grid7cd_40_oracle():
    s = workloads.grid7_cd(40)
    Fo, pp, pr, pv = oracle_factor(s)
    Xo = OL.solve(Fo, s.rhs)
    return s, pp, pr, pv, Xo


def _candidates_40():
    from paper_2512_04389_b300 import tune as T
    out = []
    for prec in ("fp64", "fp32"):
        for c in T.candidates("irregular", 64000):
            out.append((prec, dict(c)))
        for c in T.candidates("regular"):
            out.append((prec, dict(c, blocking="regular", regular_block=128)))
    return out


@pytest.mark.parametrize(
    "prec,opts", _candidates_40(),
    ids=[f"{p}-" + "-".join(f"{k}{v}" for k, v in sorted(o.items()))
         for p, o in _candidates_40()])
def test_grid7cd_40_every_tuner_candidate_against_oracle(grid7cd_40_oracle,
                                                         prec, opts):
    """Full size, n = 64,000, 4 RHS: pattern bit-exact; FP64 factors
    element-wise within 1e-10 of the oracle's and solutions within 1e-10
    (backward error <= 1e-13); FP32 factors' error reported (<= 1e-4) and
    the refined solve at backward error <= 1e-14."""
    s, pp, pr, pv, Xo = grid7cd_40_oracle
    P, F = gpu_factor(s, precision=prec, **opts)
    e = P.export()
    assert np.array_equal(e["colptr"], pp) and np.array_equal(e["rowidx"], pr)
    err = factor_error(P, F, pv)
    X, info = F.solve(_dev(s.rhs), info=True)
    Xg = X.cpu().numpy()
    xerr = np.abs(Xg - Xo).max() / np.abs(Xo).max()
    be = OL.backward_error(s.n, s.colptr, s.rowidx, s.values, Xg, s.rhs)
    print(f"{prec} {opts}: factor error {err:.2e}, solution error {xerr:.2e},"
          f" backward error {be:.2e} ({info['iterations']} refinement steps)")
    if prec == "fp64":
        assert err <= FP64_TOL and xerr <= 1e-10 and be <= 1e-13
    else:
        assert err <= 1e-4 and be <= 1e-14 and info["backward_error"] <= 1e-14


# --- failure statuses reached on the host side of the ABI

def test_refinement_not_converged_status():
    """FP32 factors, one refinement step, an unreachable tolerance:
    SLU_ERR_NOT_CONVERGED (5), X holding the last iterate."""
    s = workloads.grid7_cd(10, nrhs=2)
    P, F = gpu_factor(s, b_min=8, precision="fp32", refine_max_iter=1,
                      refine_tol=1e-300)
    with pytest.raises(S.SluError) as ei:
        F.solve(_dev(s.rhs))
    assert ei.value.status == 5
    X, info = F.solve(_dev(s.rhs), info=True, allow_not_converged=True)
    assert not info["converged"] and info["iterations"] == 1
    be = OL.backward_error(s.n, s.colptr, s.rowidx, s.values,
                           X.cpu().numpy(), s.rhs)
    assert be == pytest.approx(info["backward_error"], rel=1e-9)
    assert be <= 1e-12          # the last iterate is still a refined solution


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nonfinite_values_are_invalid(bad):
    """A NaN or infinite entry of A is SLU_ERR_INVALID_ARG (1) from
    slu_factor, and from slu_refactor when info is requested."""
    s = workloads.grid5(12)
    v = s.values.copy()
    v[v.size // 2] = bad
    P = S.Plan(s.n, s.colptr, s.rowidx, b_min=4)
    with pytest.raises(S.SluError) as ei:
        S.Factor(P, _dev(v))
    assert ei.value.status == 1 and "NaN or infinite" in str(ei.value)
    F = S.Factor(P, _dev(s.values))
    with pytest.raises(S.SluError) as ei:
        F.refactor(_dev(v), sync_info=True)
    assert ei.value.status == 1
    F.refactor(_dev(s.values), sync_info=True)        # usable again
    X = F.solve(_dev(s.rhs))
    be = OL.backward_error(s.n, s.colptr, s.rowidx, s.values,
                           X.cpu().numpy(), s.rhs)
    assert be <= 1e-13


def test_fp32_schur_tile_modes_refine_to_full_accuracy():
    """FP32 factors whose dense Schur tiles run as 3xTF32 or one TF32 pass
    on the tensor cores, or on the FP32 pipe with zero sub-tiles skipped:
    the factor error against the oracle is reported (one TF32 pass keeps 10
    mantissa bits, so it is the largest), and refinement reaches backward
    error <= 1e-14 in every mode."""
    s = workloads.grid7_cd(16, nrhs=2)
    Fo, pp, pr, pv = oracle_factor(s)
    errs = {}
    for passes in (3, 1, 0):
        P, F = gpu_factor(s, precision="fp32", dense_threshold=0.0, b_min=16,
                          tc_passes=passes)
        errs[passes] = factor_error(P, F, pv)
        X, info = F.solve(_dev(s.rhs), info=True)
        be = OL.backward_error(s.n, s.colptr, s.rowidx, s.values,
                               X.cpu().numpy(), s.rhs)
        print(f"tc_passes {passes}: factor error {errs[passes]:.2e}, "
              f"{info['iterations']} refinement steps, backward error {be:.2e}")
        assert be <= 1e-14 and info["converged"]
    assert errs[3] <= 1e-4 and errs[0] <= 1e-4 and errs[1] <= 1e-2


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_general_matrix_through_the_front_end(prec):
    """A 12^3 operator with rows and columns scrambled independently and
    rescaled over six orders of magnitude cannot be factored without row
    exchanges as given; the front end (matching + scaling + nested
    dissection, slu_reorder) makes it factorable, and the solution mapped
    back (slu_permute_scale) solves the original system."""
    from conftest import dense_to_csc
    s = workloads.grid7_cd(12, nrhs=1)
    rng = np.random.default_rng(8)
    p, q = rng.permutation(s.n), rng.permutation(s.n)
    d1, d2 = 10.0 ** rng.uniform(-3, 3, s.n), 10.0 ** rng.uniform(-3, 3, s.n)
    A = (d1[:, None] * s.dense() * d2[None, :])[np.ix_(p, q)]
    cp, ri, vx = dense_to_csc(A)
    x_true = rng.standard_normal(s.n)
    b = A @ x_true
    R = S.Reordering(s.n, cp, ri, vx, scale=True, order=True)
    rcp, rri, rvx = R.matrix()
    P, F = gpu_factor(workloads.SparseSystem(s.n, rcp, rri, rvx, np.zeros((s.n, 1))),
                      precision=prec, b_min=16)
    y, info = F.solve(R.rhs(_dev(b)), info=True)
    x = R.solution(y).cpu().numpy()
    be = OL.backward_error(s.n, cp, ri, vx, x, b)
    err = np.abs(x - x_true).max() / np.abs(x_true).max()
    print(f"{prec}: backward error {be:.2e} (original system), solution error {err:.2e}, "
          f"{info['iterations']} refinement steps")
    # the scrambled system's row and column scales span 10^6, so a backward
    # error near 1e-14 allows a larger forward error after FP32 refinement
    assert be <= 1e-13 and err <= (1e-9 if prec == "fp64" else 1e-6)
