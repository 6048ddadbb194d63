"""Device analysis (slu_analyze_device, slu_analyze_batch_device): the
symbolic factorization, Algorithm 2 and the sampling with Algorithm 3 on the
GPU must give the host analysis's plan exactly (equal plan digests, equal
exported pattern, blockptr and ptr), over the workloads, every blocking
mode, the Algorithm 3 parameters, unsorted and nonsymmetric input patterns
and the edge cases (n = 1, a single dense column, empty batch members).
The host plan itself is pinned to the oracle in test_plan_parity."""
import numpy as np
import pytest

import workloads
from conftest import random_sym_pattern

S = pytest.importorskip("paper_2512_04389_b300.slu")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _same(n, colptr, rowidx, **opts):
    h = S.Plan(n, colptr, rowidx, **opts)
    d = S.Plan(n, colptr, rowidx, device=True, **opts)
    assert d.digest() == h.digest()
    he, de = h.export(), d.export()
    assert he.keys() == de.keys()
    for k in he:
        assert np.array_equal(he[k], de[k]), k
    for k in ("nnz_sym", "nnz_lu", "flops", "nblocks_1d", "nlevels", "samples"):
        assert d.info[k] == h.info[k], k
    return h, d


def _shuffled_rows(n, colptr, rowidx, seed):
    """The same pattern with the rows of every column in random order."""
    rng = np.random.default_rng(seed)
    ri = rowidx.copy()
    for j in range(n):
        a, b = colptr[j], colptr[j + 1]
        ri[a:b] = ri[a:b][rng.permutation(b - a)]
    return ri


CASES = [
    ("grid7cd_12", lambda: workloads.grid7_cd(12)),
    ("grid5_30", lambda: workloads.grid5(30)),
    ("theta_10", lambda: workloads.grid7_theta(10)),
    ("grid5_25_natural", lambda: workloads.grid5(25, order="natural")),
]

OPTS = [
    {},
    {"dense_threshold": 0.0, "sample_points": 2000, "b_min": 8, "max_num": 1},
    {"sample_points": 37, "step": 3, "stride": 2, "max_num": 2, "b_min": 4},
    {"sample_points": 10, "step": 1, "stride": 3, "max_num": 0, "b_min": 1},
    {"blocking": 1, "regular_block": 48},
    {"blocking": 2},
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("opts", OPTS, ids=[str(i) for i in range(len(OPTS))])
def test_device_plan_equals_host_plan(name, make, opts):
    s = make()
    _same(s.n, s.colptr, s.rowidx, **opts)


@pytest.mark.parametrize("n,density,seed", [(1, 1.0, 0), (2, 0.5, 1), (57, 0.05, 2),
                                            (200, 0.02, 3), (300, 0.3, 4)])
def test_device_plan_on_random_patterns(n, density, seed):
    """Nonsymmetric patterns with unsorted rows, a missing diagonal and a
    dense column: the device symmetrizes and sorts on its own."""
    rng = np.random.default_rng(seed)
    M = rng.random((n, n)) < density
    np.fill_diagonal(M, rng.random(n) < 0.7)
    if n > 3:
        M[:, n // 2] = True                        # one dense column
    cols, rows = np.nonzero(M.T)
    colptr = np.zeros(n + 1, np.int64)
    np.add.at(colptr, cols + 1, 1)
    colptr = np.cumsum(colptr)
    rowidx = _shuffled_rows(n, colptr, rows.astype(np.int32), seed)
    _same(n, colptr, rowidx, b_min=1, sample_points=max(1, n // 3))


def test_device_plan_with_shuffled_rows():
    s = workloads.grid7_cd(10)
    ri = _shuffled_rows(s.n, s.colptr, s.rowidx, 7)
    h, d = _same(s.n, s.colptr, ri, dense_threshold=0.3)
    ref = S.Plan(s.n, s.colptr, s.rowidx, dense_threshold=0.3)
    assert h.digest() != ref.digest()               # the input order is kept
    for k in ("blockptr", "ptr", "colptr", "rowidx"):
        assert np.array_equal(h.export()[k], ref.export()[k]), k


def test_device_analysis_of_a_symmetric_random_pattern(rng):
    M = random_sym_pattern(400, 0.01, rng)
    cols, rows = np.nonzero(M.T)
    colptr = np.zeros(401, np.int64)
    np.add.at(colptr, cols + 1, 1)
    _same(400, np.cumsum(colptr), rows.astype(np.int32), b_min=2)


@pytest.mark.parametrize("opts", [{}, {"blocking": 2}, {"dense_threshold": 0.0, "b_min": 8}])
def test_device_batch_plan_equals_host_batch_plan(opts):
    ms = workloads.batch_grid5(count=12, seed=3, k_lo=4, k_hi=30)
    ns = [m.n for m in ms]
    cps = [m.colptr for m in ms]
    ris = [m.rowidx for m in ms]
    h = S.Plan(ns, cps, ris, **opts)
    d = S.Plan(ns, cps, ris, device=True, **opts)
    assert d.digest() == h.digest()


def test_device_batch_with_an_empty_member():
    a = workloads.grid5(6)
    e_cp = np.zeros(1, np.int64)
    e_ri = np.zeros(0, np.int32)
    ns = [a.n, 0, a.n]
    cps = [a.colptr, e_cp, a.colptr]
    ris = [a.rowidx, e_ri, a.rowidx]
    h = S.Plan(ns, cps, ris, b_min=2)
    d = S.Plan(ns, cps, ris, device=True, b_min=2)
    assert d.digest() == h.digest()


def test_device_analysis_on_a_side_stream():
    s = workloads.grid5(20)
    st = torch.cuda.Stream()
    h = S.Plan(s.n, s.colptr, s.rowidx)
    d = S.Plan(s.n, s.colptr, s.rowidx, device=True, stream=st)
    assert d.digest() == h.digest()


def test_device_analysis_rejects_bad_patterns_like_the_host():
    cp = np.array([0, 2, 3], np.int64)
    for ri in (np.array([0, 5, 1], np.int32), np.array([1, 1, 0], np.int32)):
        with pytest.raises(S.SluError) as eh:
            S.Plan(2, cp, ri)
        with pytest.raises(S.SluError) as ed:
            S.Plan(2, cp, ri, device=True)
        assert eh.value.status == ed.value.status == 1


def test_factor_from_a_device_plan():
    """A device plan factors and solves exactly as the host plan does."""
    s = workloads.grid7_cd(10)
    xs = []
    for dev in (False, True):
        P = S.Plan(s.n, s.colptr, s.rowidx, device=dev, dense_threshold=0.0)
        F = S.Factor(P, torch.as_tensor(s.values, device="cuda"))
        xs.append(F.solve(torch.as_tensor(s.rhs, device="cuda")).cpu().numpy())
    assert np.array_equal(xs[0], xs[1])
    r = s.dense() @ xs[1] - s.rhs
    assert np.abs(r).max() <= 1e-10 * np.abs(s.rhs).max()


@pytest.mark.parametrize("name", ["grid7cd_40", "circuit_200k"])
def test_device_analysis_at_full_size(name):
    """The bench workloads: equal digests, and the device phases reported."""
    if name == "grid7cd_40":
        s = workloads.grid7_cd(40)
        opts = {"dense_threshold": 0.0, "sample_points": 2000, "b_min": 32, "max_num": 1}
    else:
        s = workloads.circuit_bbd()
        opts = {"dense_threshold": 0.02, "sample_points": 2000, "b_min": 128, "max_num": 1}
    h = S.Plan(s.n, s.colptr, s.rowidx, **opts)
    d = S.Plan(s.n, s.colptr, s.rowidx, device=True, **opts)
    assert d.digest() == h.digest()
    print(name, "host", h.info["analyze_ms"], h.info["phase_ms"])
    print(name, "device", d.info["analyze_ms"], d.info["phase_ms"])
    hs = h.info["phase_ms"]["symbolic"] + h.info["phase_ms"]["blocking"]
    ds = d.info["phase_ms"]["symbolic"] + d.info["phase_ms"]["blocking"]
    assert ds < hs
